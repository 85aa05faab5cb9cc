"""Seeded sweep over shapes and plan options through the C ABI.

Each case draws a generator, a precision form, a storage mode, a block size,
a dimension D (every size next to a tile, chunk or block edge first, then
random sizes up to 1500) and a vector count (1..20, so every compiled
vector bucket and its padding is reached), applies the plan, then applies it
again with another vector count (the workspace is re-sized or reused), and
compares both products with the oracle within the bar of the form:

* FP64 form: 1e-12 of max|y| (summation order only);
* FP32 form: 2e-5 of max|y| against the oracle product of the FP32-form
  entries (FP32 tile sums);
* BF16X2 form: 2e-5 of max|y| against the oracle's split product.

Fixed-size tests pin each kernel; this sweep is there for index and
workspace mistakes at sizes nobody picked by hand.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EDGE_D = [2, 3, 15, 16, 17, 31, 33, 127, 128, 129, 255, 256, 257, 383, 511, 513, 1023, 1025]
NVECS = [1, 1, 2, 3, 4, 5, 6, 7, 8, 9, 11, 12, 13, 16, 17, 20]


def _cases(n=54, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        D = EDGE_D[i] if i < len(EDGE_D) else int(rng.integers(2, 1501))
        gen = int(rng.integers(0, 2))
        prec = int(rng.integers(0, 3))
        storage = int(rng.integers(0, 3))
        nvec = int(rng.choice(NVECS))
        nvec2 = int(rng.choice(NVECS))
        out.append((i, gen, prec, storage, D, nvec, nvec2))
    return out


@pytest.fixture(scope="module")
def mf():
    import paper_2606_31598_gb300 as mf
    mf.lib()
    return mf


def _make_plan(mf, gen, prec, storage, D, nvec):
    """Storage modes with an explicit 128 block so a partial cache exists
    whenever D spans two blocks; full caches get room for every pair."""
    eb = 16 if prec == 0 else 8
    nblk = (D + 127) // 128
    npair = nblk * (nblk + 1) // 2
    if storage == 1 and npair < 2:
        storage = 2
    if storage == 0:
        return mf.Plan(D, gen, seed=11, block=0, precision=prec, storage=mf.MF_STORE_PROCEDURAL, nvec_hint=nvec)
    budget = eb * 128 * 128 * (npair if storage == 2 else max(1, npair // 3))
    st = mf.MF_STORE_FULL if storage == 2 else mf.MF_STORE_PARTIAL
    return mf.Plan(D, gen, seed=11, block=128, cache_budget_bytes=budget, precision=prec, storage=st, nvec_hint=nvec)


def _reference(gen, prec, D, X):
    op = O.make_op(gen, D, seed=11, form=O.FORM_FP64 if prec == 0 else O.FORM_FP32)
    if prec == 2:
        H32 = O.window_native(O.make_op(gen, D, seed=11, form=O.FORM_FP32), 0, 0, D, D)
        return O.apply_bf16x2(O.make_op(gen, D, seed=11), X, H32)
    return O.apply(op, X)


@pytest.mark.parametrize("case", _cases(), ids=lambda c: "c%d-g%d-p%d-s%d-D%d-v%d-v%d" % c)
def test_sweep_apply_matches_oracle(mf, case):
    _, gen, prec, storage, D, nvec, nvec2 = case
    p = _make_plan(mf, gen, prec, storage, D, nvec)
    bar = 1e-12 if prec == 0 else 2e-5
    for k, nv in enumerate((nvec, nvec2)):
        X = W.random_state(D, nv, seed=100 + k)
        X = X.reshape(D, nv)
        x = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        y = torch.empty_like(x)
        p.apply(y, x, nv)
        torch.cuda.synchronize()
        p.sync()
        Y = y.cpu().numpy()
        ref = _reference(gen, prec, D, X)
        err = float(np.max(np.abs(Y - ref)) / np.max(np.abs(ref)))
        assert err < bar, (nv, err)
    p.close()


def _cheb_cases(n=16, seed=77):
    rng = np.random.default_rng(seed)
    out = []
    edges = [2, 129, 513]
    for i in range(n):
        D = edges[i] if i < len(edges) else int(rng.integers(2, 901))
        out.append((i, int(rng.integers(0, 2)), int(rng.integers(0, 2)), int(rng.integers(0, 3)), D,
                    int(rng.choice(NVECS)), float(rng.uniform(0.2, 1.0))))
    return out


@pytest.mark.parametrize("case", _cheb_cases(), ids=lambda c: "c%d-g%d-p%d-s%d-D%d-v%d-t%.2f" % c)
def test_sweep_chebyshev_matches_oracle(mf, case):
    """One Chebyshev step of exp(-i dt H) (Sec. VII) at drawn shapes; dt is
    capped so R dt <= 8 (a few tens of terms) and the oracle runs the same
    recurrence on the same form's entries with the plan's bounds."""
    _, gen, prec, storage, D, nvec, dt = case
    p = _make_plan(mf, gen, prec, storage, D, nvec)
    emin, emax = p.bounds()
    c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
    dt = min(dt, 8.0 / R)
    nt = p.cheb_terms(dt)
    X = W.random_state(D, nvec, seed=5).reshape(D, nvec)
    d = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    p.cheb_propagate(d, nvec, dt, nt)
    torch.cuda.synchronize()
    got = d.cpu().numpy()
    op = O.make_op(gen, D, seed=11, form=O.FORM_FP64 if prec == 0 else O.FORM_FP32)
    ref = O.cheb_step(op, X, dt, c, R, nt)
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert err < (1e-11 if prec == 0 else 2e-5), err
    p.close()


def _slice_cases(n=12, seed=99):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        D = int(rng.integers(129, 1501))
        ntile = -(-D // 128)
        world = int(rng.integers(2, min(4, ntile) + 1))
        out.append((i, int(rng.integers(0, 2)), int(rng.integers(0, 2)), D, world, int(rng.choice(NVECS))))
    return out


@pytest.mark.parametrize("case", _slice_cases(), ids=lambda c: "c%d-g%d-p%d-D%d-w%d-v%d" % c)
def test_sweep_row_slices_reassemble_the_product(mf, case):
    """Row-slice plans (row-parallel mode of Sec. IV.H) at drawn sizes and
    rank counts, every other slice with a partial cache of its block pairs:
    the slices' products stacked are the oracle's product."""
    from paper_2606_31598_gb300 import rowgroup
    _, gen, prec, D, world, nvec = case
    eb = 16 if prec == 0 else 8
    X = W.random_state(D, nvec, seed=6).reshape(D, nvec)
    xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    parts = []
    for k, (r0, r1) in enumerate(rowgroup.slices(D, world)):
        budget = eb * 128 * 128 * 2 if k % 2 else 0
        p = mf.Plan(D, gen, seed=11, block=128, precision=prec, cache_budget_bytes=budget,
                    storage=mf.MF_STORE_PARTIAL if budget else mf.MF_STORE_PROCEDURAL, row_begin=r0, row_end=r1)
        y = torch.empty((r1 - r0, nvec), dtype=torch.complex128, device="cuda")
        p.apply(y, xd, nvec)
        torch.cuda.synchronize()
        parts.append(y.cpu().numpy())
        p.close()
    got = np.concatenate(parts)
    ref = O.apply(O.make_op(gen, D, seed=11, form=O.FORM_FP64 if prec == 0 else O.FORM_FP32), X)
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert err < (1e-12 if prec == 0 else 2e-5), err


def _herm(rng, n):
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return 0.5 * (M + M.conj().T)


def _sysbath_cases(n=12, seed=7):
    rng = np.random.default_rng(seed)
    edges = [2, 129, 255]
    out = []
    for i in range(n):
        d_B = edges[i] if i < len(edges) else int(rng.integers(2, 901))
        out.append((i, int(rng.integers(1, 17)), d_B, int(rng.integers(0, 4)), int(rng.integers(0, 2))))
    return out


@pytest.mark.parametrize("case", _sysbath_cases(), ids=lambda c: "c%d-dS%d-dB%d-n%d-p%d" % c)
def test_sweep_sysbath_matches_oracle(mf, case):
    """System-bath plans (Sec. VII composite) at drawn d_S, d_B and numbers
    of coupling terms, against the oracle's matrix-free statement."""
    _, d_S, d_B, n_int, prec = case
    rng = np.random.default_rng(d_S * 1000 + d_B)
    H_S = _herm(rng, d_S)
    A = np.stack([_herm(rng, d_S) for _ in range(n_int)]) if n_int else np.zeros((0, d_S, d_S))
    seeds = [31 + 7 * k for k in range(n_int + 1)]
    g = 0.3
    p = mf.Plan.sysbath(d_S, d_B, seeds, H_S, A, g, precision=prec)
    X = rng.standard_normal((d_B, d_S)) + 1j * rng.standard_normal((d_B, d_S))
    ref = O.sysbath_apply(d_S, d_B, seeds, H_S, A, g, X, form=O.FORM_FP64 if prec == 0 else O.FORM_FP32)
    xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    yd = torch.empty_like(xd)
    p.apply(yd, xd, d_S)
    torch.cuda.synchronize()
    err = float(np.max(np.abs(yd.cpu().numpy() - ref)) / np.max(np.abs(ref)))
    assert err < (1e-12 if prec == 0 else 2e-5), err
    p.close()


def _external_cases(n=12, seed=8):
    rng = np.random.default_rng(seed)
    edges = [2, 128, 257]
    out = []
    for i in range(n):
        D = edges[i] if i < len(edges) else int(rng.integers(2, 1201))
        b = int(rng.choice([128, 256]))
        if b > -(-D // 128) * 128:
            b = 128  # the block may not exceed D rounded up to the tile
        nblk = -(-D // b)
        npair = nblk * (nblk + 1) // 2
        out.append((i, D, b, int(rng.integers(0, npair + 1)), int(rng.integers(0, 3)), int(rng.choice(NVECS)),
                    int(rng.choice(NVECS))))
    return out


@pytest.mark.parametrize("case", _external_cases(), ids=lambda c: "c%d-D%d-b%d-k%d-p%d-v%d-v%d" % c)
def test_sweep_external_blocks_match_dense_product(mf, case):
    """Externally stored blocks (Sec. II) at drawn sizes, block sizes and
    numbers of pairs copied to HBM (the rest read from host memory), every
    precision form, two vector counts per plan, against the dense product of
    the assembled blocks."""
    _, D, b, kpairs, prec, nvec, nvec2 = case
    rng = np.random.default_rng(D + 17 * b)
    M = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    H = (M + M.conj().T) / np.sqrt(8.0 * D)
    nblk = -(-D // b)
    P = np.zeros((nblk * b, nblk * b), dtype=np.complex128)
    P[:D, :D] = H
    dt = np.complex128 if prec == 0 else np.complex64
    blocks = np.ascontiguousarray(
        np.stack([P[n * b:(n + 1) * b, m * b:(m + 1) * b] for n, m in O.external_pairs(D, b)]).astype(dt))
    eb = 16 if prec == 0 else 8
    p = mf.Plan.external(D, b, blocks, cache_budget_bytes=kpairs * eb * b * b, precision=prec)
    assert p.describe()["pairs_cached"] == kpairs
    Hd = O.external_dense(D, b, blocks)
    bar = {0: 1e-12, 1: 2e-5, 2: 1e-4}[prec]
    for k, nv in enumerate((nvec, nvec2)):
        X = rng.standard_normal((D, nv)) + 1j * rng.standard_normal((D, nv))
        xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        yd = torch.empty_like(xd)
        p.apply(yd, xd, nv)
        torch.cuda.synchronize()
        ref = Hd @ X
        err = float(np.max(np.abs(yd.cpu().numpy() - ref)) / np.max(np.abs(ref)))
        assert err < bar, (nv, err)
    p.close()


def _filter_cases(n=8, seed=12):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        D = [2, 129][i] if i < 2 else int(rng.integers(2, 1201))
        out.append((i, int(rng.integers(0, 2)), int(rng.integers(0, 2)), int(rng.integers(0, 3)), D,
                    int(rng.choice(NVECS)), i % 2))
    return out


@pytest.mark.parametrize("case", _filter_cases(), ids=lambda c: "c%d-g%d-p%d-s%d-D%d-v%d-n%d" % c)
def test_sweep_imaginary_time_filter(mf, case):
    """exp(-tau (H - E_min)) at drawn shapes (tau so that R tau <= 6), with
    and without per-column renormalisation, against the oracle's recurrence
    with the plan's bounds.  Bars relative to the input as in the filter
    tests (divided by the smallest filtered column norm when normalised)."""
    _, gen, prec, storage, D, nvec, normalize = case
    p = _make_plan(mf, gen, prec, storage, D, nvec)
    emin, emax = p.bounds()
    c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
    tau = 6.0 / R
    nt = O.cheb_imag_terms(R * tau, 1e-15)
    op = O.make_op(gen, D, seed=11, form=O.FORM_FP64 if prec == 0 else O.FORM_FP32)
    psi = W.random_state(D, nvec, seed=9).reshape(D, nvec)
    raw = O.cheb_imag_step(op, psi, tau, c, R, nt, normalize=False).reshape(D, nvec)
    d = torch.from_numpy(np.ascontiguousarray(psi)).cuda()
    p.cheb_filter(d, nvec, tau, nt, bool(normalize))
    torch.cuda.synchronize()
    out = d.cpu().numpy().reshape(D, nvec)
    tol = (1e-13 if prec == 0 else 1e-5) * np.max(np.abs(psi))
    ref = raw
    if normalize:
        ref = raw / np.linalg.norm(raw, axis=0)
        tol /= np.min(np.linalg.norm(raw, axis=0))
        assert np.max(np.abs(np.linalg.norm(out, axis=0) - 1)) < 1e-12
    assert np.max(np.abs(out - ref)) < tol
    p.close()


def _batch_cases(n=6, seed=21):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        k = int(rng.integers(2, 7))
        Ds = [int(d) for d in rng.integers(2, 1201, k)]
        if i == 0:
            Ds[0] = 2
        nv = [int(v) for v in rng.integers(1, 17, k)]
        out.append((i, int(rng.integers(0, 2)), int(rng.integers(0, 2)), int(rng.integers(0, 2)), tuple(Ds), tuple(nv)))
    return out


@pytest.mark.parametrize("case", _batch_cases(), ids=lambda c: "c%d-g%d-p%d-full%d" % c[:4])
def test_sweep_batched_problems(mf, case):
    """Batches of 2..6 problems of drawn D (from 2) and vector counts, all
    generated or all fully cached, one Chebyshev step each in one persistent
    launch per term: every problem against the oracle's recurrence with its
    own plan's bounds and the batch's common term count."""
    _, gen, prec, full, Ds, nv = case
    # the budget is shared in proportion to D^2; a full cache of a small
    # problem still takes whole 128 x 128 blocks, so give room to spare (the
    # plans allocate only the blocks they hold)
    budget = int(1e12) if full else 0
    b = mf.Batch(list(Ds), list(nv), list(range(len(Ds))), gen, cache_budget_bytes=budget, precision=prec,
                 storage=mf.MF_STORE_FULL if full else mf.MF_STORE_PROCEDURAL)
    parts = [W.random_state(D, k, seed=40 + i).reshape(D, k) for i, (D, k) in enumerate(zip(Ds, nv))]
    d = torch.from_numpy(np.concatenate([q.ravel() for q in parts])).cuda()
    dt = 0.5 if gen == 0 else 2e-3
    nt = b.propagate(d, dt, 1)
    torch.cuda.synchronize()
    out = d.cpu().numpy()
    for i, (D, k) in enumerate(zip(Ds, nv)):
        h = b.plan(i)
        if full:
            assert mf.mf_plan_describe(h)["storage"] == "full"
        emin, emax = mf.mf_spectral_bounds(h)
        c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
        op = O.make_op(gen, D, seed=i, form=O.FORM_FP64 if prec == 0 else O.FORM_FP32)
        ref = O.cheb_step(op, parts[i], dt, c, R, nt)
        got = out[b.offsets[i]:b.offsets[i + 1]].reshape(D, k)
        assert np.max(np.abs(got - ref)) < (1e-11 if prec == 0 else 3e-5), i
    b.close()
