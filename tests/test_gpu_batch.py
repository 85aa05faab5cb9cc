"""Batched independent problems in one persistent launch per term, captured in
a CUDA graph: every problem's slice must match its own plan's propagation
and the oracle's recurrence."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mf():
    import paper_2606_31598_gb300 as mf
    mf.lib()
    return mf


@pytest.mark.parametrize("cache", ["none", "partial", "full"])
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 3e-5)])
def test_batch_matches_per_problem_and_oracle(mf, prec, tol, cache):
    """Generated chunks (no cache), a mix of stored and generated block
    pairs (partial) and stored pairs only (full); ragged D leaves a partial
    last chunk of columns and a partial last row tile."""
    # (a partial cache needs at least two block pairs: no D = 130 there)
    Ds = [1000, 2048, 700, 130 if cache != "partial" else 1200, 1536, 900]
    nv = [1, 3, 16, 2, 5, 9]
    seeds = [0, 1, 2, 3, 4, 5]
    eb = 16 if prec == 0 else 8
    full = sum(eb * D * D for D in Ds)  # every block pair, with headroom
    budget = {"none": 0, "partial": full // 5, "full": 4 * full}[cache]
    b = mf.Batch(Ds, nv, seeds, mf.MF_GEN_PHILOX_GUE, cache_budget_bytes=budget, precision=prec,
                 storage={"none": mf.MF_STORE_PROCEDURAL, "partial": mf.MF_STORE_PARTIAL,
                          "full": mf.MF_STORE_FULL}[cache])
    # FP32 problems of 1-6 vectors take the Hermitian-reuse form (each stored
    # or generated canonical chunk applied as H and as H^dagger), the others
    # the row-owner form
    assert [b.hermitian(i) for i in range(len(Ds))] == [prec == 1 and k <= 6 for k in nv]
    cached = [mf.mf_plan_describe(b.plan(i))["pairs_cached"] for i in range(len(Ds))]
    npair = [mf.mf_plan_describe(b.plan(i))["n_pair"] for i in range(len(Ds))]
    if cache == "none":
        assert sum(cached) == 0
    elif cache == "full":
        assert cached == npair
    else:
        assert any(0 < c < n for c, n in zip(cached, npair)), (cached, npair)
    total = int(b.offsets[-1])
    rng = np.random.default_rng(0)
    parts = [W.random_state(D, k, seed=10 + i).reshape(D, k) for i, (D, k) in enumerate(zip(Ds, nv))]
    packed = np.concatenate([p.ravel() for p in parts])
    assert packed.size == total
    d = torch.from_numpy(packed.copy()).cuda()
    dt, nsteps = 0.6, 2
    nt = b.propagate(d, dt, nsteps)
    nt2 = b.propagate(d, dt, nsteps)  # graph replay: two more steps
    torch.cuda.synchronize()
    assert nt == nt2 and nt > 2
    out = d.cpu().numpy()
    for i, (D, k) in enumerate(zip(Ds, nv)):
        got = out[b.offsets[i]:b.offsets[i + 1]].reshape(D, k)
        h = b.plan(i)
        emin, emax = mf.mf_spectral_bounds(h)
        c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
        H = O.dense(O.make_op(O.GEN_PHILOX_GUE, D, seed=seeds[i], form=O.FORM_FP64 if prec == 0 else O.FORM_FP32))
        ref = parts[i].copy()
        for _ in range(2 * nsteps):
            ref = O.cheb_step_dense(H, ref, dt, c, R, nt)
        assert np.max(np.abs(got - ref)) < tol, (i, np.max(np.abs(got - ref)))


def test_batch_dvr_and_workload_draw(mf):
    """DVR problems and the uneven-problem recipe (a slice of it)."""
    probs = W.batch_problems(256)
    Ds = [p[0] for p in probs[:6]]
    nv = [p[1] for p in probs[:6]]
    assert all(1024 <= D <= 32768 and D % 128 == 0 for D, _, _ in probs)
    assert all(1 <= k <= 16 for _, k, _ in probs)
    b = mf.Batch(Ds, nv, list(range(6)), mf.MF_GEN_SINC_DVR_HO, precision=mf.MF_PREC_FP64)
    n_items, grid = b.info()
    assert n_items == sum((D + 127) // 128 for D in Ds) and grid > 0
    parts = [W.random_state(D, k, seed=i).reshape(D, k) for i, (D, k) in enumerate(zip(Ds, nv))]
    d = torch.from_numpy(np.concatenate([p.ravel() for p in parts])).cuda()
    b.propagate(d, 1e-4, 1, 12)
    torch.cuda.synchronize()
    out = d.cpu().numpy()
    for i, (D, k) in enumerate(zip(Ds, nv)):
        got = out[b.offsets[i]:b.offsets[i + 1]].reshape(D, k)
        h = b.plan(i)
        emin, emax = mf.mf_spectral_bounds(h)
        c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
        ref = O.cheb_step(O.make_op(O.GEN_SINC_DVR_HO, D), parts[i], 1e-4, c, R, 12)
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-11


@pytest.mark.parametrize("cache", ["none", "full"])
def test_batch_dvr_fp32_both_forms(mf, cache):
    """DVR problems in the FP32 form: 1-6 vectors on the Hermitian-reuse form
    (real symmetric entries: H^dagger = H^T), 8, 10, 12 and 14 on the row-owner form (10 and 14
    on the batch's own 10- and 14-wide tiles); ragged
    D (a partial last chunk and row tile), generated or stored chunks."""
    Ds = [1000, 300, 1536, 777, 640, 520, 260]
    nv = [1, 6, 4, 12, 8, 10, 14]
    full = sum(8 * D * D for D in Ds)
    b = mf.Batch(Ds, nv, list(range(7)), mf.MF_GEN_SINC_DVR_HO, precision=mf.MF_PREC_FP32,
                 cache_budget_bytes=0 if cache == "none" else 4 * full,
                 storage=mf.MF_STORE_PROCEDURAL if cache == "none" else mf.MF_STORE_FULL)
    assert [b.hermitian(i) for i in range(7)] == [True, True, True, False, False, False, False]
    parts = [W.random_state(D, k, seed=20 + i).reshape(D, k) for i, (D, k) in enumerate(zip(Ds, nv))]
    d = torch.from_numpy(np.concatenate([p.ravel() for p in parts])).cuda()
    b.propagate(d, 1e-4, 1, 12)
    torch.cuda.synchronize()
    out = d.cpu().numpy()
    for i, (D, k) in enumerate(zip(Ds, nv)):
        got = out[b.offsets[i]:b.offsets[i + 1]].reshape(D, k)
        emin, emax = mf.mf_spectral_bounds(b.plan(i))
        c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
        ref = O.cheb_step(O.make_op(O.GEN_SINC_DVR_HO, D, form=O.FORM_FP32), parts[i], 1e-4, c, R, 12)
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 2e-5, (i, np.max(np.abs(got - ref)))
