"""The learned temporal predictor inside the registration: the objective is the
judge (a learned proposal is kept only where it lowers eq. (1) at the start of
the next temporal level, or over all frames for the fill after eq. (3)), and a
network trained on fields the method produced gains over the method without
it on held-out sequences."""
import numpy as np
import pytest

from _util import cuda_lib
from oracle import Params as OP
from oracle import multilevel
from paper_2001_06613_gb300 import predictor_training as PT
from paper_2001_06613_gb300 import synthetic

pytestmark = pytest.mark.gpu

# Each judged start is guaranteed an objective no higher than the classical
# start (asserted below); the final objective is not: the objective of eq. (1)
# is non-convex and Gauss-Newton runs to its stopping tests from different
# starts, which end in different local minima.  Measured on GB300 with the
# GIRs running to their tolerances: within 2 % on these sequences (4 % at
# paper scale).  The gain at equal final objective is measured by bench.py
# (target objective), not asserted here.
FINAL_J_SPREAD = 5e-2

TRAIN_SEEDS = list(range(100, 108))
HELD_OUT = [200, 201, 202]


@pytest.fixture(scope="module")
def S():
    return cuda_lib()


def _params(S, **kw):
    return S.stml_default_params(n_levels=2, n_tlevels=2, **kw)


def _register(S, R, net=None, **kw):
    import torch
    ctx = S.Context(_params(S, **kw))
    try:
        S.stml_load_sequence(ctx.ptr, torch.from_numpy(R).cuda())
        S.stml_build_pyramid(ctx.ptr)
        if net is not None:
            S.stml_set_predictor_net(ctx, net)
        stats = S.stml_register(ctx.ptr, 0)
        y = np.empty((R.shape[0], 2) + R.shape[1:], np.float32)
        S.stml_get_field(ctx.ptr, 1, y)
        return y, stats, ctx.params
    finally:
        ctx.close()


def _final_J(R, y, prm):
    op = OP(alpha=prm.alpha, alpha_t=prm.alpha_t, lam=prm.lambda_, beta=prm.beta)
    return multilevel.final_objective(R.astype(np.float64), y.astype(np.float64), op)["J"]


def test_judge_keeps_the_lower_objective(S):
    """An untrained network with a random head: every proposal is judged, the
    start of each GIR is the lower of the two objectives, and the result stays
    a valid registration."""
    R = synthetic.make_sequence(synthetic.spec_tiny(seed=3))
    net = S.Net(synthetic.net_init_params(9, head_scale=0.5), max_batch=8, max_h=64, max_w=64)
    try:
        y, stats, prm = _register(S, R, net)
    finally:
        net.close()
    y0, stats0, _ = _register(S, R)
    judged = [s for s in stats if s["pred_learned"] >= 0]
    assert judged, "no learned proposal was judged"
    for s in judged:
        assert s["J0"] <= s["J0_classic"] * (1 + 1e-6) + 1e-12
    for s in stats:
        if s["fill_learned"] >= 0:
            assert s["J_fill"] <= s["J_fill_classic"]
    J, J0 = _final_J(R, y, prm), _final_J(R, y0, prm)
    print(f"\nrandom-head network: decisions {[s['pred_learned'] for s in stats]}, final J {J:.6g} vs {J0:.6g}")
    assert abs(J - J0) <= FINAL_J_SPREAD * J0


def test_zero_head_network_changes_nothing_on_the_coarsest_level(S):
    """With a zero head the network proposes linear interpolation: on the
    coarsest level that is the classical predictor itself, so the objective
    ties and the classical proposal is kept."""
    R = synthetic.make_sequence(synthetic.spec_tiny(seed=4))
    net = S.Net(synthetic.net_init_params(10), max_batch=8, max_h=64, max_w=64)
    try:
        _, stats, _ = _register(S, R, net)
    finally:
        net.close()
    coarse = [s for s in stats if s["level"] == 0 and s["tlevel"] > 0]
    assert coarse and all(s["pred_learned"] == 0 for s in coarse)
    assert all(s["J0"] == s["J0_classic"] for s in coarse)


def test_trained_network_gains_on_held_out_sequences(S):
    """Trained on fields the method produced for 8 sequences; on 3 held-out
    sequences of the same kind the trained network predicts the registered
    fields better than interpolation (the untrained network), and the
    registration with it starts the corrections from lower objectives."""
    prm = _params(S)
    train_R = [synthetic.make_sequence(synthetic.spec_tiny(seed=s)) for s in TRAIN_SEEDS]
    test_R = [synthetic.make_sequence(synthetic.spec_tiny(seed=s)) for s in HELD_OUT]
    data = PT.collect(S, train_R, prm)
    held = PT.collect(S, test_R, prm)
    net = S.Net(synthetic.net_init_params(11), max_batch=16, max_h=64, max_w=64)
    try:
        before = PT.mean_loss(S, net, held, batch=16, crop=32)
        losses = PT.train(S, net, data, steps=400, batch=16, crop=32, lr=5e-4, seed=1, log_every=100)
        after = PT.mean_loss(S, net, held, batch=16, crop=32)
        rows = []
        for R in test_R:
            y, st, p = _register(S, R, net)
            y0, st0, _ = _register(S, R)
            rows.append((st, st0, _final_J(R, y, p), _final_J(R, y0, p)))
    finally:
        net.close()
    print(f"\ntraining loss {losses}; held-out loss (cells^2): interpolation {before:.4g}, trained {after:.4g}")
    for st, st0, J, J0 in rows:
        cg, cg0 = sum(s["cg_iters"] for s in st), sum(s["cg_iters"] for s in st0)
        gn, gn0 = sum(s["gn_iters"] for s in st), sum(s["gn_iters"] for s in st0)
        kept = [s["pred_learned"] for s in st]
        starts = [(round(s["J0"], 6), round(s["J0_classic"], 6)) for s in st if s["pred_learned"] >= 0]
        print(f"  learned kept {kept}; starts (learned-or-kept, classical) {starts}; PCG iterations {cg} vs "
              f"{cg0}; GN {gn} vs {gn0}; final J {J:.6g} vs {J0:.6g}")
        assert abs(J - J0) <= FINAL_J_SPREAD * J0
        for s in st:
            if s["pred_learned"] >= 0:
                assert s["J0"] <= s["J0_classic"] * (1 + 1e-6) + 1e-12
    assert after < before
