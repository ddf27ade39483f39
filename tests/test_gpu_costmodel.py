"""GPU tests of the learned cost model: the forward pass and the gradient of the library's
own kernels against the float64 oracle, training on measured item durations, and what the
trained network gains over the wedge-share order of the work queue, and over Algorithm 4's
fanout order, on graphs it was not trained on.
"""

from __future__ import annotations

import heapq

import numpy as np
import pytest

from oracle import costmodel as cm
from paper_2601_17707_gb300 import bbc, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _away_from_kinks(p, X, margin=1e-3):
    """Rows whose hidden pre-activations all sit farther than `margin` from 0, so that
    float32 and float64 take the same ReLU branches."""
    _, (_, z1, _, z2, _, _) = cm.forward(p, X)
    return (np.abs(z1).min(axis=1) > margin) & (np.abs(z2).min(axis=1) > margin)


def test_forward_and_gradient_match_the_oracle(gpu_lib):
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.3, cm.N_PARAMS).astype(np.float32)
    X = rng.uniform(0, 1.5, (6000, cm.KF)).astype(np.float32)
    X = X[_away_from_kinks(p.astype(np.float64), X.astype(np.float64))][:4096]
    t = rng.normal(0, 1, X.shape[0]).astype(np.float32)
    m = bbc.CostModel(seed=1)
    m.set_params(p)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    # fp32 sums of at most 33 products per unit: 1e-4 relative is a wide margin
    y = m.predict(Xd).cpu().numpy()
    y_ref, _ = cm.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.allclose(y, y_ref, rtol=1e-4, atol=1e-4 * np.abs(y_ref).max())
    L, g = m.loss_grad(Xd, td)
    L_ref, g_ref = cm.grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert L == pytest.approx(L_ref, rel=1e-4)
    # per-sample gradients summed over 4,096 samples in fp32 (per-lane sums, then atomics)
    scale = np.abs(g_ref).max()
    assert np.abs(g.astype(np.float64) - g_ref).max() <= 2e-4 * scale
    # the parameters round-trip
    assert np.array_equal(m.get_params(), p)


def test_training_steps_match_the_oracle(gpu_lib):
    """bbc_cost_model_fit against oracle.costmodel.fit: the standardised log-cycle labels
    (through the loss at the starting parameters) and the parameters after 1 and after
    10 full-batch Adam steps (Kingma and Ba's update with bias correction), element by
    element. Tolerance: at lr = 1e-4 a parameter moves at most 1e-3 in 10 steps; float32
    gradients (relative error ~1e-5) change each normalised step by about that fraction of
    lr, so 5e-6 absolute leaves a wide margin, while a missing bias correction (a first
    step 3.16 lr long) or a wrong moment update misses it by two orders of magnitude."""
    rng = np.random.default_rng(21)
    n = 4096
    X = rng.uniform(0, 1.5, (n, cm.KF)).astype(np.float32)
    cycles = np.exp(6.0 + 1.5 * X[:, 0] - 0.7 * X[:, 2] + 0.3 * X[:, 5] * X[:, 6]
                    + 0.1 * rng.normal(size=n)).astype(np.int64)
    p0 = rng.normal(0, 0.3, cm.N_PARAMS).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    cd = torch.from_numpy(cycles).cuda()
    X64 = X.astype(np.float64)
    for steps in (1, 10):
        m = bbc.CostModel(seed=3)
        m.set_params(p0)                     # also clears the moments
        L0 = m.fit(Xd, cd, steps=0, lr=1e-4)
        t_ref, _, _ = cm.standardised_labels(cycles)
        assert L0 == pytest.approx(cm.loss(p0.astype(np.float64), X64, t_ref), rel=1e-4)
        L = m.fit(Xd, cd, steps=steps, lr=1e-4)
        p_ref, L_ref, _ = cm.fit(p0.astype(np.float64), X64, cycles, steps=steps, lr=1e-4)
        got = m.get_params().astype(np.float64)
        err = np.abs(got - p_ref)
        assert err.max() <= 5e-6, (steps, int(err.argmax()), float(err.max()))
        assert L == pytest.approx(L_ref, rel=1e-4)
        m.free()


def _fanout(g, side):
    """Algorithm 4's queue key on pair side S: fanout(u) = sum over v in N(u) of deg(v),
    plus deg(u)."""
    s_ids, c_ids = (g.u, g.v) if side == 0 else (g.v, g.u)
    n_s, n_c = (g.n_u, g.n_v) if side == 0 else (g.n_v, g.n_u)
    deg_s = np.bincount(s_ids, minlength=n_s).astype(np.int64)
    deg_c = np.bincount(c_ids, minlength=n_c).astype(np.int64)
    return np.bincount(s_ids, weights=deg_c[c_ids], minlength=n_s).astype(np.int64) + deg_s


def _items(g):
    G = bbc.Graph.from_synthetic(g)
    X = G.item_features()
    c = G.item_cycles()
    return G, X, c


def test_training_reduces_the_loss(gpu_lib):
    G, X, c = _items(synth.powerlaw_1m_200k(seed=11, scale=0.1))
    try:
        assert X.shape[0] == c.shape[0] > 1000
        assert bool((c > 0).all())
        m = bbc.CostModel(seed=0)
        start = m.fit(X, c, steps=0)
        end = m.fit(X, c, steps=500, lr=3e-3)
        assert end < 0.5 * start and end < 0.5      # standardised labels: variance 1
    finally:
        G.free()


def test_item_anchors_match_the_degree_feature(gpu_lib):
    g = synth.powerlaw_1m_200k(seed=12, scale=0.05)
    G = bbc.Graph.from_synthetic(g)
    try:
        X = G.item_features().cpu().numpy().astype(np.float64)
        a = G.item_anchors().cpu().numpy().astype(np.int64)
        side = G.info().side
        s_ids, n_s = (g.u, g.n_u) if side == 0 else (g.v, g.n_v)
        assert a.shape[0] == X.shape[0] > 0 and a.min() >= 0 and a.max() < n_s
        deg = np.bincount(s_ids, minlength=n_s).astype(np.float64)
        assert np.allclose(X[:, 1], np.log1p(deg[a]) / 16.0, rtol=1e-6, atol=1e-6)
    finally:
        G.free()


def _spearman(a, b):
    ra = np.argsort(np.argsort(a)).astype(np.float64)
    rb = np.argsort(np.argsort(b)).astype(np.float64)
    return float(np.corrcoef(ra, rb)[0, 1])


def _makespan(order, cost, workers):
    """Greedy list schedule, items in `order` to the first free worker: what the
    persistent queue does."""
    heap = [0.0] * workers
    for i in order:
        heapq.heapreplace(heap, heap[0] + float(cost[i]))
    return max(heap)


def test_what_the_learned_model_gains_over_the_wedge_estimate(gpu_lib):
    """Trained on the item durations of five graphs, evaluated on a sixth. The queue's
    own estimate of an item's cost is its share of the anchor's wedges (feature 7). The
    network's gain is in predicting the cost itself: its held-out error in log cycles is
    compared with the best affine map of the wedge share (least squares on the same
    training items). Ordering the queue by either gives the same makespan here (the
    wedge share already ranks items almost perfectly, and even the true costs leave
    under 1 % to gain): the network gains nothing for the schedule, which the test
    reports and bounds in both directions. The paper's own order, by each anchor's
    fanout (Algorithm 4), is simulated beside them."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    Xs, cs = [], []
    for seed, scale in ((21, 0.05), (22, 0.08), (23, 0.12), (24, 0.15)):
        G, X, c = _items(synth.powerlaw_1m_200k(seed=seed, scale=scale))
        Xs.append(X)
        cs.append(c)
        G.free()
    G, X, c = _items(synth.hubs_50k_2m(seed=5, scale=0.01))
    Xs.append(X)
    cs.append(c)
    G.free()
    X_train, c_train = torch.cat(Xs), torch.cat(cs)
    m = bbc.CostModel(seed=0)
    m.fit(X_train, c_train, steps=800, lr=3e-3)
    log_train = np.log(np.maximum(c_train.cpu().numpy(), 1).astype(np.float64))
    mu, sd = log_train.mean(), log_train.std()
    share_train = X_train[:, 7].cpu().numpy().astype(np.float64)
    A = np.stack([share_train, np.ones_like(share_train)], axis=1)
    coef, *_ = np.linalg.lstsq(A, log_train, rcond=None)

    g = synth.powerlaw_1m_200k(seed=31, scale=0.1)          # not seen in training
    G, X, c = _items(g)
    try:
        cost = c.cpu().numpy().astype(np.float64)
        log_test = np.log(np.maximum(cost, 1))
        pred = m.predict(X).cpu().numpy().astype(np.float64) * sd + mu    # log cycles
        share = X[:, 7].cpu().numpy().astype(np.float64)
        lin = coef[0] * share + coef[1]
        mse_model = float(np.mean((pred - log_test) ** 2))
        mse_share = float(np.mean((lin - log_test) ** 2))
        rho_model, rho_share = _spearman(pred, cost), _spearman(share, cost)
        workers = 2 * sms
        ms_share = _makespan(np.argsort(-share, kind="stable"), cost, workers)
        ms_model = _makespan(np.argsort(-pred, kind="stable"), cost, workers)
        ms_best = _makespan(np.argsort(-cost, kind="stable"), cost, workers)
        # Algorithm 4: the items of each anchor in decreasing fanout of the anchor
        fan = _fanout(g, G.info().side)[G.item_anchors().cpu().numpy().astype(np.int64)]
        ms_fanout = _makespan(np.argsort(-fan, kind="stable"), cost, workers)
        print(f"held-out log-cycle MSE: network {mse_model:.4f}, affine wedge share {mse_share:.4f}; "
              f"rank correlation: network {rho_model:.3f}, wedge share {rho_share:.3f}; "
              f"simulated makespan (cycles): fanout order {ms_fanout:.4g}, wedge order {ms_share:.4g}, "
              f"learned {ms_model:.4g}, true-cost order {ms_best:.4g}")
        # what the network gains: a better cost prediction ...
        assert mse_model < mse_share
        assert rho_model > rho_share - 0.02
        # ... and no scheduling gain: the learned order's makespan is the wedge order's
        # (and the fanout order's) to within 2 %, either way. Real tile-kernel times with
        # the learned order against the default order showed no gain either (measured,
        # not asserted here: 18.31 against 18.34 ms on the 20M-edge graph, 28.2-29.0
        # against 28.3 ms on the 100M-edge heavy-hub graph).
        assert abs(ms_model - ms_share) <= 0.02 * ms_share
        assert abs(ms_model - ms_fanout) <= 0.02 * ms_fanout
        # the real queue with the learned order: same counts
        before = G.count()[:2]
        m.order(G)
        assert G.count()[:2] == before
    finally:
        G.free()
