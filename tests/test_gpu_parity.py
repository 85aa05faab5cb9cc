"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Bars: generated entries bit-exact per precision form; products within the
relative errors derived from the arithmetic (FP64 form: 1e-12 of max|y|,
accumulation order only; FP32 form against the oracle product of the same
FP32-form entries: 2e-5 of max|y|, FP32 tile sums of up to D terms); the
FP32 form's deviation from the FP64 operator is reported and bounded.
"""
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


def _plan(mf, D, gen, prec, seed=1, block=0, budget=0, storage=None, **kw):
    opts = {"precision": prec}
    if storage is not None:
        opts["storage"] = storage
    opts.update(kw)
    return mf.Plan(D, gen, seed=seed, block=block, cache_budget_bytes=budget, **opts)


def _form(prec):
    return O.FORM_FP64 if prec == 0 else O.FORM_FP32


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _apply(plan, x):
    xd = _dev(x)
    yd = torch.empty_like(xd)
    plan.apply(yd, xd, 1 if x.ndim == 1 else x.shape[1])
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _relerr(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# --------------------------------------------------------------- entries ----
@pytest.mark.parametrize("prec", [0, 1])
def test_gue_entries_bit_exact(mf, prec):
    D = 1000
    p = _plan(mf, D, mf.MF_GEN_PHILOX_GUE, prec, seed=7)
    op = O.make_op(O.GEN_PHILOX_GUE, D, seed=7, form=_form(prec))
    for (r0, c0, rows, cols) in [(0, 0, 64, 64), (500, 300, 40, 90), (937, 0, 63, 1000), (0, 999, 1000, 1)]:
        g = p.entries(r0, c0, rows, cols)
        ref = O.window(op, r0, c0, rows, cols) if prec == 0 else O.window_native(op, r0, c0, rows, cols)
        assert g.dtype == ref.dtype
        assert np.array_equal(g.view(np.uint8), ref.view(np.uint8)), (r0, c0)


@pytest.mark.parametrize("prec", [0, 1])
def test_dvr_entries_bit_exact(mf, prec):
    D = 131072
    p = _plan(mf, D, mf.MF_GEN_SINC_DVR_HO, prec)
    op = O.make_op(O.GEN_SINC_DVR_HO, D, form=_form(prec))
    for (r0, c0, rows, cols) in [(0, 0, 32, 32), (70000, 3, 8, 40), (5, 131000, 16, 72)]:
        g = p.entries(r0, c0, rows, cols)
        ref = O.kinetic_window(op, r0, c0, rows, cols)
        if prec == 0:
            assert np.array_equal(g.real, ref) and np.all(g.imag == 0)
        else:
            assert np.array_equal(g.real, ref.astype(np.float32)) and np.all(g.imag == 0)


def test_entries_partition_invariant(mf):
    """Entries come from global (row, col): any block size gives the same H."""
    D = 700
    a = _plan(mf, D, mf.MF_GEN_PHILOX_GUE, 1, block=128).entries(0, 0, D, D)
    b = _plan(mf, D, mf.MF_GEN_PHILOX_GUE, 1, block=512).entries(0, 0, D, D)
    assert np.array_equal(a.view(np.uint8), b.view(np.uint8))


# --------------------------------------------------------------- products ----
@pytest.mark.parametrize("gen", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("D,block", [(4096, 512), (1000, 256), (129, 0), (2, 0)])
def test_apply_matches_oracle(mf, gen, prec, D, block):
    p = _plan(mf, D, gen, prec, seed=1, block=block)
    x = W.random_state(D, 1, seed=1)
    y = _apply(p, x)
    op = O.make_op(gen, D, seed=1, form=_form(prec))
    ref = O.apply(op, x, block=block)
    tol = 1e-12 if prec == 0 else 2e-5
    assert _relerr(y, ref) < tol
    if prec == 1:
        # stated error of the FP32 form against the FP64 operator
        ref64 = O.apply(O.make_op(gen, D, seed=1), x, block=block)
        assert _relerr(y, ref64) < (2e-4 if gen == 0 else 5e-3)


@pytest.mark.parametrize("prec", [0, 1])
def test_dvr_full_size_sampled_rows(mf, prec):
    """Workload size D = 131072 in the benchmark's launch shape; 24 sampled
    output rows computed by the oracle one by one (ragged tail included)."""
    D = 131072
    p = _plan(mf, D, mf.MF_GEN_SINC_DVR_HO, prec)
    x = W.wavepacket(D)
    y = _apply(p, x)
    rows = np.array([0, 1, 511, 512, 4095, 4096, 65535, 65536, 65700, 66000, 70000, 90001,
                     100000, 120000, 131000, 131070, 131071, 2048, 8191, 16384, 32767, 65600, 65800, 66100])
    op = O.make_op(O.GEN_SINC_DVR_HO, D, form=_form(prec))
    ref = O.apply_rows(op, x, rows)[:, 0]
    scale = np.max(np.abs(O.apply_rows(O.make_op(O.GEN_SINC_DVR_HO, D), x, rows)))
    err = np.max(np.abs(y[rows] - ref)) / scale
    assert err < (1e-11 if prec == 0 else 2e-3)


@pytest.mark.parametrize("prec", [0, 1])
def test_dvr_full_size_every_row_against_fft(mf, prec):
    """D = 131072 in the benchmark's launch shape, every output row against
    the oracle's FFT form of the Toeplitz product (FP64 reference of the
    FP64 form, or of the FP32 form's entries)."""
    D = 131072
    p = _plan(mf, D, mf.MF_GEN_SINC_DVR_HO, prec)
    rng = np.random.default_rng(11)
    x = (rng.standard_normal(D) + 1j * rng.standard_normal(D)) / np.sqrt(2.0 * D)
    y = _apply(p, x)
    ref = O.dvr_apply_fft(O.make_op(O.GEN_SINC_DVR_HO, D, form=_form(prec)), x)
    # a random x has no cancellation: the FP32 tile sums hold 2e-5 of max|y|
    assert _relerr(y, ref) < (1e-11 if prec == 0 else 2e-5)


def test_hermitian_identity_on_gpu(mf):
    D = 2048
    p = _plan(mf, D, 0, 0, seed=3)
    x = W.random_state(D, 1, seed=4)
    z = W.random_state(D, 1, seed=5)
    lhs = np.vdot(x, _apply(p, z))
    rhs = np.vdot(_apply(p, x), z)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# ----------------------------------------------------------------- cache ----
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("gen", [0, 1])
def test_cache_modes_bit_identical(mf, prec, gen):
    """Procedural, partial and full caching apply the same entries in the same
    order: the products agree bit for bit (Sec. III.A: caching must not change H)."""
    D, b = 1000, 256
    eb = 16 if prec == 0 else 8
    x = W.random_state(D, 1, seed=2)
    ys, kinds = [], []
    for storage, budget in [(mf.MF_STORE_PROCEDURAL, 0), (mf.MF_STORE_PARTIAL, 3 * b * b * eb),
                            (mf.MF_STORE_FULL, 10 * b * b * eb)]:
        p = _plan(mf, D, gen, prec, block=b, budget=budget, storage=storage)
        desc = p.describe()
        kinds.append((desc["storage"], desc["pairs_cached"]))
        ys.append(_apply(p, x))
    if gen == 1:
        # the DVR's procedural path is the Toeplitz-window kernel: compare the
        # two cached forms bitwise and the procedural one within tolerance
        assert np.array_equal(ys[1], ys[2])
        assert _relerr(ys[0], ys[2]) < (1e-12 if prec == 0 else 2e-5)
    else:
        assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[1], ys[2])
    assert kinds == [("procedural", 0), ("partial", 3), ("full", 10)]


# ------------------------------------------------------------- Chebyshev ----
@pytest.mark.parametrize("prec", [0, 1])
def test_cheb_step_matches_oracle_gue(mf, prec):
    """D = 4096 Philox ensemble, 32 terms, t = 1 (the small workload)."""
    D = 4096
    p = _plan(mf, D, 0, prec, seed=1, block=512)
    emin, emax = p.bounds()
    op = O.make_op(O.GEN_PHILOX_GUE, D, seed=1, form=_form(prec))
    H = O.dense(op)
    E = np.linalg.eigvalsh(H)
    assert emin < E[0] and E[-1] < emax  # Lanczos bounds enclose the spectrum
    psi = W.random_state(D, 1, seed=1)
    dpsi = _dev(psi)
    p.cheb_propagate(dpsi, 1, 1.0, 32)
    torch.cuda.synchronize()
    out = dpsi.cpu().numpy()
    c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
    ref = O.cheb_step_dense(H, psi, 1.0, c, R, 32)
    assert np.max(np.abs(out - ref)) < (1e-11 if prec == 0 else 2e-5)
    assert abs(np.linalg.norm(out) - 1) < (1e-12 if prec == 0 else 1e-5)
    if prec == 0:
        w, V = np.linalg.eigh(H)
        exact = V @ (np.exp(-1j * w) * (V.conj().T @ psi))
        assert np.max(np.abs(out - exact)) < 1e-11


def test_cheb_dvr_half_period_closed_form(mf):
    """Harmonic oscillator: psi(pi)(x) = -i psi0(-x) for the coherent state."""
    D = 256
    p = _plan(mf, D, 1, 0, cheb_tol=1e-14)
    psi0 = W.wavepacket(D)
    d = _dev(psi0)
    nsteps = 40
    for _ in range(nsteps):
        p.cheb_propagate(d, 1, np.pi / nsteps, 0)
    torch.cuda.synchronize()
    out = d.cpu().numpy()
    assert np.max(np.abs(out - (-1j) * psi0[::-1])) < 1e-8


def test_cheb_terms_rule(mf):
    D = 4096
    p = _plan(mf, D, 0, 0, seed=1, block=512)
    emin, emax = p.bounds()
    R = 0.5 * (emax - emin)
    for dt in (0.1, 1.0, 7.0):
        assert p.cheb_terms(dt) == O.cheb_terms(R * dt, 1e-7)


# ------------------------------------------------------------ edge cases ----
def test_bad_calls_rejected(mf):
    D = 300
    p = _plan(mf, D, 0, 1)
    x = _dev(W.random_state(D, 1))
    with pytest.raises(mf.MFError):
        p.apply(x, x, 1)  # aliasing
    with pytest.raises(mf.MFError):
        p.apply(torch.empty_like(x), x, 0)
    with pytest.raises(mf.MFError):
        p.cheb_propagate(x, 1, -1.0, 8)
    with pytest.raises(mf.MFError):
        p.set_bounds(1.0, 0.0)


# --------------------------------------------------------- multi-vector ----
@pytest.mark.parametrize("gen", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nvec", [2, 3, 16, 32, 64])
def test_multivector_apply_matches_oracle(mf, gen, prec, nvec):
    """Y = H X (Eq. generic_multivector) by the row-owner kernels, ragged D."""
    D = 1000
    p = _plan(mf, D, gen, prec, seed=5, block=256)
    X = W.random_state(D, nvec, seed=7)
    Y = _apply(p, X)
    ref = O.apply(O.make_op(gen, D, seed=5, form=_form(prec)), X, block=256)
    assert _relerr(Y, ref) < (1e-12 if prec == 0 else 2e-5)


@pytest.mark.parametrize("prec", [0, 1])
def test_multivector_row_owner_and_hermitian_reuse_agree(mf, prec):
    """The row-owner kernel (hermitian_reuse = 0) and the Hermitian-reuse
    kernel give the oracle's product (ragged D, 5 vectors, cached and
    generated block pairs)."""
    D, nvec = 1000, 5
    op = O.make_op(O.GEN_PHILOX_GUE, D, seed=3, form=_form(prec))
    X = W.random_state(D, nvec, seed=8).reshape(D, nvec)
    ref = O.apply(op, X)
    eb = 16 if prec == 0 else 8
    for reuse in (0, -1):
        p = _plan(mf, D, 0, prec, seed=3, block=256, budget=3 * eb * 256 * 256, storage=mf.MF_STORE_PARTIAL,
                  hermitian_reuse=reuse, nvec_hint=nvec)
        y = _apply(p, X)
        assert _relerr(y, ref) < (1e-12 if prec == 0 else 2e-5)


@pytest.mark.parametrize("prec,nvec", [(0, 8), (1, 8), (1, 32), (1, 64)])
def test_multivector_cache_modes_bit_identical(mf, prec, nvec):
    """Generated, partially and fully cached block pairs give the same
    product bit for bit (8 vectors: the Hermitian-reuse kernel; 32 and 64 in
    the FP32 form: the row-owner ring tile, stored chunks read in both
    orientations)."""
    D, b = 1000, 256
    eb = 16 if prec == 0 else 8
    X = W.random_state(D, nvec, seed=3)
    ys = []
    for storage, budget in [(mf.MF_STORE_PROCEDURAL, 0), (mf.MF_STORE_PARTIAL, 4 * b * b * eb),
                            (mf.MF_STORE_FULL, 10 * b * b * eb)]:
        ys.append(_apply(_plan(mf, D, 0, prec, block=b, budget=budget, storage=storage), X))
    assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2])


@pytest.mark.parametrize("gen,storage", [(0, 0), (0, 1), (0, 2), (1, 2)])
def test_two_vectors_on_the_tile_kernel(mf, gen, storage):
    """Two vectors in the FP32 form run on the canonical-tile kernel with both
    vectors in registers: every column equals the one-vector product bit for
    bit (same operations in the same order), generated, partially cached and
    fully cached (and stored DVR blocks) alike, and matches the oracle; the
    row-owner kernel agrees within the form's tolerance."""
    D, b = 1000, 256
    budget = {0: 0, 1: 4 * b * b * 8, 2: 10 * b * b * 8}[storage]
    X = W.random_state(D, 2, seed=14).reshape(D, 2)
    p = _plan(mf, D, gen, 1, seed=6, block=b, budget=budget, storage=storage, nvec_hint=2)
    assert p.describe()["path"] == "herm_tile"
    Y = _apply(p, X)
    for v in range(2):
        assert np.array_equal(Y[:, v], _apply(p, np.ascontiguousarray(X[:, v])))
    ref = O.apply(O.make_op(gen, D, seed=6, form=O.FORM_FP32), X)
    assert _relerr(Y, ref) < 2e-5
    q = _plan(mf, D, gen, 1, seed=6, block=b, budget=budget, storage=storage, nvec_hint=2, hermitian_reuse=0)
    assert _relerr(_apply(q, X), Y) < 2e-5


def test_multivector_matches_single_vector_columns(mf):
    """Each column of the multi-vector product equals the one-vector product."""
    D, nvec = 700, 5
    p = _plan(mf, D, 0, 0, seed=2)
    X = W.random_state(D, nvec, seed=9)
    Y = _apply(p, X)
    for v in range(nvec):
        assert _relerr(Y[:, v], _apply(p, np.ascontiguousarray(X[:, v]))) < 1e-13


@pytest.mark.parametrize("prec", [0, 1])
def test_multivector_cheb_matches_oracle(mf, prec):
    D, nvec = 1024, 4
    p = _plan(mf, D, 0, prec, seed=4, block=512)
    emin, emax = p.bounds()
    H = O.dense(O.make_op(O.GEN_PHILOX_GUE, D, seed=4, form=_form(prec)))
    X = W.random_state(D, nvec, seed=11)
    d = _dev(X)
    p.cheb_propagate(d, nvec, 0.7, 24)
    torch.cuda.synchronize()
    out = d.cpu().numpy()
    c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
    ref = O.cheb_step_dense(H, X, 0.7, c, R, 24)
    assert np.max(np.abs(out - ref)) < (1e-11 if prec == 0 else 2e-5)


def test_generator_division_and_sqrt_exact_on_this_gpu(mf):
    """The FP32 generator's Markstein-corrected division and square root equal
    IEEE round-to-nearest on every float of their input ranges."""
    assert mf.mf_selfcheck_generator() == (0, 0)


@pytest.mark.parametrize("nvec", [1, 3])
@pytest.mark.parametrize("imag", [False, True])
def test_dvr_fp32_chebyshev_terms_against_oracle(mf, imag, nvec):
    """FP32 DVR plans, real- and imaginary-time Chebyshev steps through the
    window kernels: D = 10000 spans three 4096-row tiles with a ragged last
    one (one vector) or five 2048-row tiles (3 vectors, padded to 4); the
    oracle runs the same recurrence on the same FP32-form entries in FP64."""
    D = 10000
    p = _plan(mf, D, mf.MF_GEN_SINC_DVR_HO, 1, nvec_hint=nvec)
    emin, emax = p.bounds()
    c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
    op = O.make_op(O.GEN_SINC_DVR_HO, D, form=O.FORM_FP32)
    psi = W.wavepacket(D) if nvec == 1 else W.random_state(D, nvec, seed=12).reshape(D, nvec)
    d = _dev(psi)
    if imag:
        tau, nt = 2e-4, 24
        p.cheb_filter(d, nvec, tau, nt, True)
        ref = O.cheb_imag_step(op, psi, tau, c, R, nt, normalize=True)
    else:
        dt, nt = 1e-4, 24
        p.cheb_propagate(d, nvec, dt, nt)
        ref = O.cheb_step(op, psi, dt, c, R, nt)
    torch.cuda.synchronize()
    out = d.cpu().numpy()
    assert np.max(np.abs(out - ref)) < 2e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("nvec", [2, 4, 5, 8, 13, 16])
def test_dvr_multivector_window_kernel(mf, nvec):
    """FP32 DVR products of 2..16 vectors by the multi-vector window kernel
    (vector buckets 2, 4, 8, 16; its row tiles are 4096 / bucket x 16 rows,
    its chunks 8192 / bucket columns): D = 5000 spans several row tiles and
    column chunks of every bucket with ragged tails.  Every column against
    the oracle's FFT form of the FP32 form's entries and against the
    one-vector kernel."""
    D = 5000
    p = _plan(mf, D, mf.MF_GEN_SINC_DVR_HO, 1, nvec_hint=nvec)
    rng = np.random.default_rng(20 + nvec)
    X = (rng.standard_normal((D, nvec)) + 1j * rng.standard_normal((D, nvec))) / np.sqrt(2.0 * D)
    Y = _apply(p, X)
    op = O.make_op(O.GEN_SINC_DVR_HO, D, form=O.FORM_FP32)
    for v in range(nvec):
        ref = O.dvr_apply_fft(op, X[:, v])
        assert _relerr(Y[:, v], ref) < 2e-5, v
        assert _relerr(Y[:, v], _apply(p, np.ascontiguousarray(X[:, v]))) < 2e-5, v


@pytest.mark.parametrize("nvec", [2, 16])
def test_dvr_multivector_full_size_against_fft(mf, nvec):
    """D = 131072 (the benchmark's grid) with 2 and 16 vectors: every row of
    the first and last columns against the oracle's FFT form."""
    D = 131072
    p = _plan(mf, D, mf.MF_GEN_SINC_DVR_HO, 1, nvec_hint=nvec)
    rng = np.random.default_rng(31)
    X = (rng.standard_normal((D, nvec)) + 1j * rng.standard_normal((D, nvec))) / np.sqrt(2.0 * D)
    Y = _apply(p, X)
    op = O.make_op(O.GEN_SINC_DVR_HO, D, form=O.FORM_FP32)
    for v in (0, nvec - 1):
        assert _relerr(Y[:, v], O.dvr_apply_fft(op, X[:, v])) < 2e-5, v
