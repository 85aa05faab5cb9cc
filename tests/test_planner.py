"""Analytic planner (Algorithm 1) and surrogate oracle pins; host only.

Expected values are the paper's printed numbers for its 18-qubit run
(Sec. VII: block 4096 = 128 MiB in complex64, 32 GiB of operator per GPU in
a two-GPU row group for two operators, 2.749e11 real FLOP per application,
20 coupling values over 4 GPU groups = 5 waves, score 5 x 0.104089 s) and the
definitions of Sec. IV (Eq. partial_cache_pairs and the memory constraint).
"""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as MO


@pytest.fixture(scope="module")
def mf():
    import paper_2606_31598_gb300 as mf
    from paper_2606_31598_gb300 import _build
    _build.build()
    return mf


def _est(mf, pr, c, budget=0.0, alpha=0.9, model=None):
    return mf.mf_planner_estimate(pr, c, model, alpha, budget)


def test_paper_18_qubit_storage_flops_and_waves(mf):
    # d_B = 2^16 bath dimension, R = d_S = 4, n_op = 2 (H_B and B_1), complex64
    pr = mf.mf_problem(2 ** 16, 2 ** 16, 4, 2, 20, 8.0, 43.97 * 2 ** 30, 8)
    c = mf.mf_candidate(4096, mf.MF_STORE_FULL, -1, 2, 4, 3)
    e = _est(mf, pr, c)
    assert e.n_blk == 16
    assert e.M_block == 128 * 2 ** 20                 # 4096^2 x 8 B
    assert e.M_op == 32 * 2 ** 30                     # 2 operators x 16 GiB row slice
    assert abs(e.F_mv - 2.749e11) / 2.749e11 < 1e-3   # 2 d_S d_B^2 8
    assert e.waves == 5                               # ceil(20 / 4)
    assert abs(e.waves * 0.104089 - 0.520447) < 5e-6  # S_bench = W t_mv
    assert e.feasible == 1
    # one 16 GiB row slice per operator: 32768 x 65536 x 8 B
    one = _est(mf, mf.mf_problem(2 ** 16, 2 ** 16, 4, 1, 1, 8.0, 1e12, 1), mf.mf_candidate(4096, 2, -1, 2, 1, 3))
    assert one.M_op == 32768 * 65536 * 8


def test_explicit_dense_sizes(mf):
    # complex64 D = 2^18: 8 D^2 = 2^39 bytes; complex128: 1 TiB
    for bc, want in [(8.0, 2 ** 39), (16.0, 2 ** 40)]:
        pr = mf.mf_problem(2 ** 18, 2 ** 18, 1, 1, 1, bc, 1e15, 1)
        e = _est(mf, pr, mf.mf_candidate(0, mf.MF_STORE_FULL, -1, 1, 1, 0))
        assert e.M_op == want and e.M_tot == want


def test_partial_cache_pairs_equation(mf):
    """P_cache = min(N_pair, floor(M_cache / (B_c b^2))) for D = 262144,
    b = 2048, 120 GB at 8 B per entry: N_pair = 128*129/2 = 8256, 3576 pairs."""
    pr = mf.mf_problem(262144, 262144, 64, 1, 1, 8.0, 280e9, 1)
    e = _est(mf, pr, mf.mf_candidate(2048, mf.MF_STORE_PARTIAL, -1, 1, 1, 4), budget=120e9)
    assert e.n_blk == 128 and e.n_pair == 8256
    assert e.pairs_cached == math.floor(120e9 / (8 * 2048 ** 2)) == 3576
    assert e.M_op == 3576 * 2048 ** 2 * 8
    # budget larger than the operator: all pairs
    e2 = _est(mf, pr, mf.mf_candidate(2048, mf.MF_STORE_PARTIAL, -1, 1, 1, 4), budget=1e15)
    assert e2.pairs_cached == 8256


def test_memory_constraint_boundary(mf):
    """Accept iff M_tot <= alpha min M_free (Eq. planner_memory_constraint)."""
    D, R, bc = 10000, 2, 8.0
    m_work = 4 * D * R * bc
    c = mf.mf_candidate(0, mf.MF_STORE_PROCEDURAL, -1, 1, 1, 4)
    ok = _est(mf, mf.mf_problem(D, D, R, 1, 1, bc, m_work / 0.9, 1), c)
    bad = _est(mf, mf.mf_problem(D, D, R, 1, 1, bc, m_work / 0.9 * (1 - 1e-9), 1), c)
    assert ok.M_work == m_work and ok.feasible == 1 and bad.feasible == 0


def test_model_score_prefers_cache_for_seeded_and_window_for_dvr(mf):
    pr = mf.mf_problem(65536, 65536, 1, 1, 1, 8.0, 200e9, 1)
    gue = mf.mf_device_model(7.4e13, 6.7e12, 4e11)
    proc = _est(mf, pr, mf.mf_candidate(2048, 0, -1, 1, 1, 4), model=gue, budget=100e9)
    full = _est(mf, pr, mf.mf_candidate(2048, 2, -1, 1, 1, 4), model=gue, budget=100e9)
    assert full.S_model < proc.S_model
    dvr = mf.mf_device_model(7.4e13, 6.7e12, 1e15)
    proc_d = _est(mf, pr, mf.mf_candidate(2048, 0, -1, 1, 1, 4), model=dvr, budget=100e9)
    full_d = _est(mf, pr, mf.mf_candidate(2048, 2, -1, 1, 1, 4), model=dvr, budget=100e9)
    assert proc_d.S_model < full_d.S_model


def test_estimate_rejects_bad_input(mf):
    import ctypes
    L = mf.lib()
    e = mf.mf_estimate()
    pr = mf.mf_problem(0, 10, 1, 1, 1, 8.0, 1e9, 1)
    c = mf.mf_candidate(0, 0, -1, 1, 1, 1)
    assert L.mf_planner_estimate(ctypes.byref(pr), ctypes.byref(c), None, 0.9, 0.0, ctypes.byref(e)) == 1
    pr = mf.mf_problem(10, 10, 1, 1, 1, 8.0, 1e9, 1)
    assert L.mf_planner_estimate(ctypes.byref(pr), ctypes.byref(c), None, 1.5, 0.0, ctypes.byref(e)) == 1


def test_features_vector(mf):
    f = mf.mf_mlp_features(0, 1, 65536, 2048, 16, 30e9)
    assert f[0] == 16 and f[1] == 11 and f[2] == 4
    assert list(f[3:8]) == [1, 0, 0, 1, 0]
    full = (32 * 33 / 2) * 8 * 2048 ** 2
    assert abs(f[8] - min(1.0, 30e9 / full)) < 1e-6
    assert abs(f[9] - math.log10(31.0)) < 1e-6


# ------------------------------------------------ surrogate oracle pins ----
def test_mlp_oracle_gradient_against_finite_differences():
    rng = np.random.default_rng(0)
    F, H, O, n = 5, 7, 3, 13
    p = rng.standard_normal(F * H + H + H * H + H + H * O + O) * 0.4
    X = rng.standard_normal((n, F))
    Y = rng.standard_normal((n, O))
    M = (rng.random((n, O)) > 0.3).astype(float)
    mu, sd = MO.zscore(X)
    _, g = MO.loss_grad(p, mu, sd, X, Y, M, F, H, O)
    h = 1e-6
    for i in rng.choice(p.size, 40, replace=False):
        e = np.zeros_like(p)
        e[i] = h
        num = (MO.loss_grad(p + e, mu, sd, X, Y, M, F, H, O)[0] - MO.loss_grad(p - e, mu, sd, X, Y, M, F, H, O)[0]) / (2 * h)
        assert abs(num - g[i]) < 1e-7 * max(1.0, abs(num))


def test_mlp_oracle_adam_fits_a_smooth_map():
    rng = np.random.default_rng(1)
    F, H, O = 3, 16, 2
    X = rng.uniform(-1, 1, (200, F))
    Y = np.stack([np.sin(X[:, 0]) + X[:, 1] ** 2, X[:, 2] * X[:, 0]], 1)
    p0 = rng.standard_normal(F * H + H + H * H + H + H * O + O) * 0.3
    mu, sd = MO.zscore(X)
    _, curve = MO.train_adam(p0, mu, sd, X, Y, None, F, H, O, 600, 1e-2)
    assert curve[-1] < 0.02 * curve[0]


# ------------------------------------------------------- sweep machinery ----
def test_sweep_candidates_follow_partial_cache_equation(mf):
    from paper_2606_31598_gb300 import planner_sweep as PS
    D, nv, budget = 131072, 16, 30e9   # canonical cache about 69 GB in the FP32 form
    cs = PS.candidates(mf, 0, mf.MF_PREC_FP32, D, nv, budget, [256, 2048, 4096])
    for c in cs:
        b = c["block"]
        nblk = -(-D // b)
        npair = nblk * (nblk + 1) // 2
        if c["storage"] == "partial":
            assert c["pairs_cached"] == min(npair, math.floor(budget / (8 * b * b)))
        if c["storage"] == "procedural":
            assert c["pairs_cached"] == 0
    assert {c["storage"] for c in cs} == {"procedural", "partial"}
    # at D = 32768 the whole canonical cache (about 4.6 GB) fits the budget
    cs2 = PS.candidates(mf, 0, mf.MF_PREC_FP32, 32768, nv, budget, [2048])
    assert {c["storage"] for c in cs2} == {"procedural", "full"}


def test_regret_definition():
    from paper_2606_31598_gb300 import planner_sweep as PS

    class Fake:  # predicts the measured log-time exactly
        def __init__(self, recs):
            self.t = {tuple(r["features"]) + (r["storage"],): r["t_mv"] for r in recs}

        def predict(self, X):
            out = np.full((len(X), 3), 1e9, np.float32)
            for i, x in enumerate(X):
                for k, st in enumerate(PS.STRATEGIES):
                    key = tuple(float(v) for v in x) + (st,)
                    if key in self.t:
                        out[i, k] = math.log(self.t[key])
            return out

    recs = []
    for p in range(4):
        for j, (st, t, sm) in enumerate([("procedural", 2.0, 1.0), ("full", 1.0, 3.0), ("partial", 1.5, 2.0)]):
            recs.append({"problem": "p%d" % p, "storage": st, "t_mv": t * (1 + p), "S_model": sm,
                         "features": [float(p), float(j)] + [0.0] * 8})
    assert PS.regret(recs, Fake(recs))["mean"] == 0.0
    an = PS.regret(recs, None)   # the model picks procedural: regret 1.0 on every problem
    assert abs(an["mean"] - 1.0) < 1e-12 and an["zero_regret_frac"] == 0.0
    tr, te = PS.split(recs, 0.25, seed=0)
    assert {r["problem"] for r in tr}.isdisjoint({r["problem"] for r in te})


def test_shipped_gb300_records_give_the_reported_analytic_regret(mf):
    """The sweep records measured on GB300 with the current kernels ship
    with the package (480-problem grid, cheapest first under a 32-minute
    cap: 475 problems, 4275 records).  They were scored at sweep time by the
    library's current Algorithm 1 (re-scoring them with mf_planner_estimate
    and mf_planner_device_model changes no score), so the analytic regret
    recomputed from them (seed-0 split of problems) is that of the ranking
    the library runs, on measurements its rates were not tuned on."""
    from paper_2606_31598_gb300 import planner_sweep as ps
    recs = ps.load(ps.RECORDS_GB300)
    assert len(recs) == 4275
    assert len({r["problem"] for r in recs}) == 475
    assert all(r["t_mv"] > 0 and len(r["features"]) == 10 for r in recs)
    assert max(abs(a["S_model"] / b["S_model"] - 1.0) for a, b in zip(ps.rescore(recs), recs)) == 0.0
    train, test = ps.split(recs, 0.2, 0)
    a_test, a_train = ps.regret(test, None), ps.regret(train, None)
    assert a_test["problems"] == 95 and a_train["problems"] == 380
    assert abs(a_test["mean"] - 0.0014020) < 1e-6 and abs(a_test["max"] - 0.026763) < 1e-5
    assert abs(a_train["mean"] - 0.0012458) < 1e-6


def _fit_oracle_surrogate(ps, MO, train, residual, epochs):
    """Algorithm 3's surrogate in the oracle's FP64 form (10 or 11 inputs ->
    64 -> 64 -> 3, masked squared loss, Adam) fitted to the records."""
    X = ps.surrogate_inputs(train, residual).astype(np.float64)
    Y = np.zeros((len(train), 3))
    M = np.zeros((len(train), 3))
    for i, r in enumerate(train):
        k = ps.STRATEGIES.index(r["storage"])
        Y[i, k] = math.log(r["t_mv"]) - (math.log(r["S_model"]) if residual else 0.0)
        M[i, k] = 1.0
    F, H, O = X.shape[1], 64, 3
    rng = np.random.default_rng(0)
    p = np.concatenate([(rng.standard_normal(F * H) / np.sqrt(F)), np.zeros(H),
                        (rng.standard_normal(H * H) / np.sqrt(H)), np.zeros(H),
                        (rng.standard_normal(H * O) / np.sqrt(H)), np.zeros(O)])
    mu, sd = MO.zscore(X)
    p, curve = MO.train_adam(p, mu, sd, X, Y, M, F, H, O, epochs=epochs, lr=3e-3)

    class Net:
        n_in = F

        def predict(self, Xq):
            return MO.forward(p, mu, sd, np.asarray(Xq, np.float64), F, H, O)[3]

    return Net(), curve


def test_learned_planners_against_the_current_algorithm_1(mf):
    """Algorithm 3 against the library's current Algorithm 1 on the fresh
    GB300 records, held out by problem.  Both surrogate forms -- direct (ln
    t_mv from the 10 features) and residual (ln S_model as an 11th input,
    learning ln t_mv - ln S_model) -- fitted for 1500 epochs in the oracle's
    FP64 form pick plans with lower mean held-out regret than Algorithm 1
    (0.11 % direct, 0.064 % residual, against 0.140 %) and a smaller largest
    miss (2.1-2.2 % against 2.7 %).  The margins are at the timing noise of
    the records: an 800-epoch fit gives 0.18 % and 0.22 %, a 3000-epoch fit
    0.15 % and 0.057 %, and the library's FP32 GPU fits (3000 epochs) 0.114 %
    and 0.116 %; so the learned planner matches the re-calibrated analytic
    one rather than beating it by a margin that would survive re-measuring.
    Against running without a planner (a fixed block of 2048 with no cache,
    or with all the cache the budget allows) the trained network's picks
    are over 100x closer to the measured best."""
    from oracle import mlp_oracle as MO
    from paper_2606_31598_gb300 import planner_sweep as ps
    train, test = ps.split(ps.load(ps.RECORDS_GB300), 0.2, 0)
    analytic = ps.regret(test, None)
    # without a planner: a fixed block of 2048, no cache (17 % mean regret,
    # up to 2.5x slower) or all the cache the budget allows (87 %, up to 11x)
    proc, cache = ps.fixed_regret(test, "procedural"), ps.fixed_regret(test, "max_cache")
    assert abs(proc["mean"] - 0.17209) < 1e-4 and abs(cache["mean"] - 0.87144) < 1e-4, (proc, cache)
    for residual, want in ((False, 0.00111), (True, 0.00064)):
        net, curve = _fit_oracle_surrogate(ps, MO, train, residual, 1500)
        assert curve[-1] < 0.002 * curve[0]
        learned = ps.regret(test, net)
        assert abs(learned["mean"] - want) < 1e-4, (residual, learned)
        assert learned["mean"] < analytic["mean"] and learned["max"] < analytic["max"], (residual, learned, analytic)
        # the gain over running without a planner: over 100x in mean regret
        assert learned["mean"] < 0.01 * min(proc["mean"], cache["mean"]), (learned, proc, cache)


def test_device_model_rejects_bad_input(mf):
    with pytest.raises(mf.MFError):
        mf.mf_planner_device_model(7, 0, 152)
    with pytest.raises(mf.MFError):
        mf.mf_planner_device_model(1, 0, 0)


@pytest.mark.parametrize("prec", [1, 2])
def test_library_model_prefers_the_cache_for_philox_vectors_and_generation_for_dvr(mf, prec):
    """With the library's runtime-model rates, 16 Philox vectors with room for
    the whole canonical cache are planned with it (measured on GB300: full
    cache about 2x faster than generation), while the DVR stays procedural
    (its window table makes generation nearly free)."""
    D, R = 65536, 16
    pr = mf.mf_problem(D, D, R, 1, 1, 8.0, 250e9, 1)
    budget = 40e9
    for gen, want_cache in ((0, True), (1, False)):
        dm = mf.mf_planner_device_model(prec, gen, 152)
        proc = _est(mf, pr, mf.mf_candidate(2048, 0, -1, 1, 1, 4), model=dm, budget=budget)
        full = _est(mf, pr, mf.mf_candidate(2048, 2, -1, 1, 1, 4), model=dm, budget=budget)
        assert (full.S_model < proc.S_model) == want_cache, (gen, full.S_model, proc.S_model)
