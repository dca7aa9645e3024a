"""The learned join-size estimator on the GPU: gradients and BF16 inference
against the float64 oracle (oracle.mlp), and the engine's predicted
single-pass joins: trained on logged joins, bit-exact fixpoints, fewer
launches than the exact count-scan-write joins, a lower prediction loss
than the estimators it learns from, and exact fallback on forced
under-prediction."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2501_13051_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cdl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2501_13051_gb300 import build as B
    B.build()
    from paper_2501_13051_gb300 import cdl as C
    return C


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def batch(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 20, size=(n, M.D_IN)).astype(np.float32)
    y = rng.uniform(0, 25, size=n).astype(np.float32)
    theta = (M.init(seed) * 0.5).astype(np.float32)
    return theta, X, y


@pytest.mark.parametrize("n,tau", [(1, 0.9), (37, 0.9), (500, 0.5), (2000, 0.1)])
def test_gradient_matches_oracle(cdl, n, tau):
    theta, X, y = batch(n, n)
    out, grad = cdl.mlp_gradient(dev(theta), dev(X), dev(y), tau)
    pred, _ = M.forward(theta.astype(np.float64), X.astype(np.float64))
    _, g = M.gradient(theta.astype(np.float64), X.astype(np.float64), y.astype(np.float64), tau)
    out, grad = out.cpu().numpy(), grad.cpu().numpy()
    assert np.all(np.abs(out - pred) <= 1e-4 * (1 + np.abs(pred)))
    # FP32 sums over <= 2000 samples of <= 64 terms: relative error well under 1e-4
    assert np.linalg.norm(grad - g) <= 1e-4 * np.linalg.norm(g)
    assert np.all(np.abs(grad - g) <= 1e-4 * np.abs(g).max() + 1e-7)
    fwd = cdl.mlp_forward(dev(theta), dev(X)).cpu().numpy()
    assert np.array_equal(fwd, out)


def test_bf16_inference(cdl):
    theta, X, y = batch(5, 300)
    got = cdl.mlp_infer_bf16(dev(theta), dev(X)).cpu().numpy()
    ref = M.forward_bf16(theta, X)
    # same roundings; only the FP32 summation order differs, which may move a
    # hidden value across a BF16 rounding boundary (one BF16 ulp, 2^-8)
    assert np.all(np.abs(got - ref) <= 2e-3 * (1 + np.abs(ref)))
    fp, _ = M.forward(theta.astype(np.float64), X.astype(np.float64))
    assert np.median(np.abs(got - fp) / (1 + np.abs(fp))) <= 0.01


def test_adam_kernel_matches_oracle(cdl):
    """k_adam over four steps (bias correction at t = 1..4, changing
    gradients) against oracle.mlp.adam in float64."""
    rng = np.random.default_rng(11)
    th = rng.normal(size=M.N_PARAMS).astype(np.float32)
    m = np.zeros(M.N_PARAMS)
    v = np.zeros(M.N_PARAMS)
    d_th, d_m, d_v = dev(th), dev(m), dev(v)
    ref = th.astype(np.float64)
    m_abs = np.zeros(M.N_PARAMS)  # the first moment's terms in magnitude
    for t in range(1, 5):
        g = (rng.normal(size=M.N_PARAMS) * 10.0 ** rng.integers(-4, 2, size=M.N_PARAMS)).astype(np.float32)
        cdl.mlp_adam(d_th, dev(g), d_m, d_v, t, 3e-3)
        ref, m, v = M.adam(ref, g.astype(np.float64), m, v, t, lr=3e-3)
        m_abs = 0.9 * m_abs + 0.1 * np.abs(g)
    got = d_th.cpu().numpy().astype(np.float64)
    # FP32 state: each step moves a parameter by at most lr, with relative
    # error ~1e-6; four steps stay well within 1e-5 of the step size
    assert np.all(np.abs(got - ref) <= 1e-6 + 1e-6 * np.abs(ref))
    # FP32 rounding relative to the terms summed (m may cancel to near 0)
    assert np.all(np.abs(d_m.cpu().numpy() - m) <= 1e-6 * m_abs + 1e-12)
    assert np.allclose(d_v.cpu().numpy(), v, rtol=1e-5, atol=1e-12)


def _feature_case(kind, rng):
    if kind == "uniform":
        return [rng.integers(0, 1 << 20, 100_000)], [np.sort(rng.integers(0, 1 << 20, 50_000))]
    if kind == "zipf":
        return [np.minimum(rng.zipf(1.3, 300_000), 1 << 30)], [np.sort(np.minimum(rng.zipf(1.1, 4000), 1 << 30))]
    if kind == "small":
        return [rng.integers(0, 50, 700)], [np.sort(rng.integers(0, 50, 33))]
    if kind == "equal":
        return [np.full(5000, 7)], [np.full(3000, 7)]
    if kind == "two-column":
        return ([rng.integers(0, 300, 9000), rng.integers(0, 5, 9000)],
                [rng.integers(0, 300, 2049), rng.integers(0, 5, 2049)])
    if kind == "empty-probe":
        return [np.zeros(0, np.int64)], [np.arange(100)]
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["uniform", "zipf", "small", "equal", "two-column",
                                  "empty-probe"])
def test_join_features_match_oracle(cdl, kind):
    """k_join_features against the float64 statement of the 16 features
    (oracle.features): distinct counts exact, the rest to FP32 rounding."""
    import torch
    from oracle import features as F
    rng = np.random.default_rng(len(kind))
    probe, build = _feature_case(kind, rng)
    probe = [np.asarray(c, dtype=np.uint32) for c in probe]
    build = [np.asarray(c, dtype=np.uint32) for c in build]
    host = (float(3 * len(probe[0]) + 1), float(len(np.unique(build[0]))), 4.0, 1234.0, 567.0,
            1.0 if kind == "small" else 0.0)
    to = lambda a: torch.from_numpy(a.view(np.int32)).cuda()
    got = cdl.join_features([to(c) for c in probe], [to(c) for c in build], host).cpu().numpy()
    want = F.join_features(probe[0], build[0], host,
                           probe_k1=probe[1] if len(probe) > 1 else None,
                           build_k1=build[1] if len(build) > 1 else None)
    assert np.all(np.abs(got - want) <= 1e-5 + 1e-5 * np.abs(want)), (got, want)
    # the distinct counts are integers on both sides
    assert np.array_equal(np.round(2.0 ** got[3:5] - 1), np.round(2.0 ** want[3:5] - 1))


def log_joins(cdl, programs):
    X, y = [], []
    for prog in programs:
        with cdl.Engine(estimator=2) as e:
            e.load_program(prog)
            e.run()
            a, b = e.estimator_log()
            X.append(a)
            y.append(b)
    return np.concatenate(X), np.concatenate(y)


def training_programs():
    progs = [W.tc_program(W.er_graph(n, m, s)) for n, m, s in
             ((300, 450, 1), (600, 900, 2), (1000, 1500, 3), (800, 1000, 4), (1500, 2000, 5))]
    progs += [W.sg_program(W.random_forest(n, s)) for n, s in ((2000, 6), (4000, 7), (8000, 8))]
    progs += [W.points_to_program(W.points_to_edb(1 / 4096, 9))]
    return progs


@pytest.fixture(scope="module")
def trained(cdl):
    X, y = log_joins(cdl, training_programs())
    assert len(y) > 100
    with cdl.Engine() as e:
        loss = e.estimator_train(X, y, epochs=3000, lr=3e-3, tau=0.9, seed=1)
        params = e.estimator_params()
    return X, y, params, loss


def test_trained_network_beats_its_inputs(cdl, trained):
    """What the network gains: its pinball loss (tau 0.9) on the logged joins
    against (a) the histogram join estimate it gets as feature 6, (b) the
    previous round's size of the same join step (feature 13) and (c) the best
    constant."""
    X, y, params, loss = trained
    tau = 0.9
    pred = cdl.mlp_infer_bf16(dev(params), dev(X)).cpu().numpy()
    l_net = M.pinball(pred, y, tau)
    l_hist = M.pinball(X[:, 6], y, tau)
    l_prev = M.pinball(X[:, 13], y, tau)
    l_const = M.pinball(np.full_like(y, np.quantile(y, tau)), y, tau)
    assert l_net < 0.8 * min(l_hist, l_prev, l_const), (l_net, l_hist, l_prev, l_const)
    assert loss == pytest.approx(M.pinball(M.forward(params.astype(np.float64), X)[0], y, tau),
                                 rel=1e-3, abs=1e-3)


@pytest.mark.parametrize("make", [lambda: W.sg_program(W.random_forest(6000, 99)),
                                  lambda: W.tc_program(W.er_graph(1200, 1700, 98)),
                                  lambda: W.points_to_program(W.points_to_edb(1 / 4096, 97))])
def test_predicted_joins_are_exact_and_cheaper(cdl, oracle_lib, trained, make):
    _, _, params, _ = trained
    prog = make()
    want = oracle_lib.run_program(prog)
    # sorted rows (dense_bits=-1): a bitmap head needs no predicted buffer
    exact, st0 = cdl.run_program(prog, dense_bits=-1)
    with cdl.Engine(estimator=1, est_params=params, est_min_rows=1, dense_bits=-1) as e:
        e.load_program(prog)
        st = e.run()
        got = {nm: e.export(nm) for nm in prog.arity}
    for nm in prog.arity:
        assert np.array_equal(got[nm], want.relations[nm]), nm
    assert st.iterations == want.iterations and st.delta_per_round == st0.delta_per_round
    assert st.est_predictions > 0
    assert st.est_overflows <= st.est_predictions  # fallbacks are the exception
    # no count pass, no scan, no offsets: the joins move fewer bytes
    assert st.algo_bytes < st0.algo_bytes


def test_forced_underprediction_falls_back_exactly(cdl, oracle_lib, trained):
    _, _, params, _ = trained
    prog = W.sg_program(W.random_forest(5000, 11))
    want = oracle_lib.run_program(prog)
    with cdl.Engine(estimator=1, est_params=params, est_margin=-40.0, est_min_rows=1,
                    dense_bits=-1) as e:
        e.load_program(prog)
        st = e.run()
        got = e.export("sg")
    assert np.array_equal(got, want.relations["sg"])
    assert st.est_overflows > 0 and st.iterations == want.iterations


def test_estimator_without_weights_is_exact(cdl, oracle_lib):
    prog = W.tc_program(W.er_graph(200, 300, 3))
    with cdl.Engine(estimator=1, est_min_rows=1) as e:
        e.load_program(prog)
        st = e.run()
        got = e.export("path")
    assert st.est_predictions == 0
    assert np.array_equal(got, oracle_lib.run_program(prog).relations["path"])


def constant_network(log2_size):
    """Parameters of a network that predicts log2_size for every join (all
    weights zero, output bias set): a prediction large enough to hold the
    join, so the single-pass path writes it."""
    p = np.zeros(cdl_params(), dtype=np.float32)
    p[-1] = log2_size
    return p


def cdl_params():
    from paper_2501_13051_gb300 import cdl as C
    return C.MLP_PARAMS


def hot_key_program(with_filter):
    # one key matches 10,000 build rows: every probe row on it is cut into
    # chunks of the single-pass join's work list
    hub = np.stack([np.full(10_000, 7), np.arange(10_000)], 1)
    hub = np.concatenate([hub, [[1, 2], [1, 3], [2, 5]]])
    src = np.stack([np.arange(30), np.where(np.arange(30) % 3 == 0, 1, 7)], 1)
    neq = (("x", "y"),) if with_filter else ()
    return W.Program(arity={"hub": 2, "src": 2, "out": 2},
                     edb={"hub": hub.astype(np.uint32), "src": src.astype(np.uint32)},
                     rules=[W.Rule(("out", ("x", "y")), (("src", ("x", "h")), ("hub", ("h", "y"))),
                                   neq)])


@pytest.mark.parametrize("with_filter", [False, True])
def test_hot_keys_through_the_single_pass_join(cdl, oracle_lib, with_filter):
    prog = hot_key_program(with_filter)
    want = oracle_lib.run_program(prog)
    with cdl.Engine(estimator=1, est_params=constant_network(20.0), est_min_rows=1,
                    dense_bits=-1) as e:
        e.load_program(prog)
        st = e.run()
        got = e.export("out")
    assert np.array_equal(got, want.relations["out"])
    assert st.est_predictions > 0 and st.est_overflows == 0


def test_dense_heads_take_no_prediction(cdl, oracle_lib):
    """A head kept as a bitmap has no buffer to size: its joins keep the
    exact count pass even with a network that predicts every join."""
    prog = hot_key_program(False)
    with cdl.Engine(estimator=1, est_params=constant_network(20.0), est_min_rows=1) as e:
        e.load_program(prog)
        st = e.run()
        got = e.export("out")
    assert np.array_equal(got, oracle_lib.run_program(prog).relations["out"])
    assert st.est_predictions == 0
