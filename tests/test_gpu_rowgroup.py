"""Row-distributed plans (row-parallel mode, Sec. IV.H) on one GPU: plans for
row slices apply H[rows, :] to the whole vector and cache only the pairs
their rows touch; slice plans stepped in lockstep (gathers emulated by
concatenation), and two processes driving rowgroup.propagate over a gloo
all-gather, give the oracle's Chebyshev step.

Bars: FP64 form 1e-12 of max|y| (summation order), FP32 form 2e-5."""
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


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("gen,prec", [(0, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("nvec", [1, 3])
def test_slices_reassemble_the_product(mf, gen, prec, nvec):
    from paper_2606_31598_gb300 import rowgroup
    D = 1000 if gen == 0 else 5000
    form = O.FORM_FP64 if prec == 0 else O.FORM_FP32
    X = W.random_state(D, nvec, seed=2).reshape(D, nvec)
    ref = O.apply(O.make_op(gen, D, seed=4, form=form), X)
    xd = torch.from_numpy(X).cuda()
    parts = []
    eb = 16 if prec == 0 else 8
    for k, (r0, r1) in enumerate(rowgroup.slices(D, 3)):
        budget = (2 * eb * 256 * 256) if k == 1 else 0   # one slice with a partial cache
        p = mf.Plan(D, gen, seed=4, block=256, precision=prec, cache_budget_bytes=budget, row_begin=r0, row_end=r1)
        if k == 1 and gen == 0:
            assert p.describe()["pairs_cached"] == 2
        y = torch.empty((r1 - r0, nvec), dtype=torch.complex128, device="cuda")
        p.apply(y, xd, nvec)
        parts.append(y)
    torch.cuda.synchronize()
    got = torch.cat(parts).cpu().numpy()
    assert _rel(got, ref) < (1e-12 if prec == 0 else 2e-5)


def _padded_bounds(op, pad=0.05):
    """Spectral bounds from the oracle's dense eigenvalues, padded by 5 % of
    the half-width (any enclosure gives the same exp(-i dt H) psi)."""
    ev = np.linalg.eigvalsh(O.dense(op))
    half = 0.5 * (ev[-1] - ev[0])
    return ev[0] - pad * half, ev[-1] + pad * half


def test_lockstep_row_group_step_matches_oracle(mf):
    """Two slice plans stepped term by term (gather = concatenation) against
    the oracle's Chebyshev step with the same bounds and term count."""
    from paper_2606_31598_gb300 import rowgroup
    D, nvec, dt = 1000, 2, 0.8
    op = O.make_op(O.GEN_PHILOX_GUE, D, seed=6)
    emin, emax = _padded_bounds(op)
    c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
    psi = W.random_state(D, nvec, seed=5).reshape(D, nvec)
    plans = []
    for r0, r1 in rowgroup.slices(D, 2):
        p = mf.Plan(D, 0, seed=6, precision=0, cheb_tol=1e-13, row_begin=r0, row_end=r1)
        p.set_bounds(emin, emax)
        plans.append(p)
    nts = [p.rows_cheb_begin(dt) for p in plans]
    assert nts[0] == nts[1] and nts[0] > 8
    nt = nts[0]
    psi_d = torch.from_numpy(psi).cuda()
    st = []
    for p in plans:
        rows = p.row_end - p.row_begin
        acc = torch.empty((rows, nvec), dtype=torch.complex128, device="cuda")
        p.rows_cheb_init(psi_d, acc, nvec)
        st.append([acc, torch.zeros_like(acc), torch.empty_like(acc)])
    q_full = psi_d
    for j in range(1, nt):
        for p, (acc, qp, qn) in zip(plans, st):
            p.rows_cheb_term(j, q_full, qp, qn, acc, nvec)
        q_full = torch.cat([s[2] for s in st])
    outs = []
    for p, (acc, _, _) in zip(plans, st):
        o = torch.empty_like(acc)
        p.rows_cheb_final(acc, o, nvec, dt)
        outs.append(o)
    torch.cuda.synchronize()
    got = torch.cat(outs).cpu().numpy()
    ref = O.cheb_step(op, psi, dt, c, R, nt)
    assert np.max(np.abs(got - ref)) < 1e-11


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, case, out):
    """One rank of a row group: its slice plan on the one GPU, the library's
    slice calls through rowgroup.propagate, a gloo all-gather of host copies
    between terms."""
    import os
    import torch.distributed as dist
    import paper_2606_31598_gb300 as mf
    from paper_2606_31598_gb300 import rowgroup
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        gen, prec, D, nvec, dt, bounds, psi = case
        r0, r1 = rowgroup.slices(D, world)[rank]
        budget = (2 * 16 * 256 * 256) if rank == 1 else 0
        p = mf.Plan(D, gen, seed=6, block=256, precision=prec, cheb_tol=1e-13, cache_budget_bytes=budget,
                    row_begin=r0, row_end=r1)
        if bounds is not None:
            p.set_bounds(*bounds)
        res = rowgroup.propagate(p, torch.from_numpy(psi).cuda(), nvec, dt,
                                 rowgroup.dist_allgather(host=True))
        torch.cuda.synchronize()
        out[rank] = (r0, r1, res.cpu().numpy(), p.describe()["pairs_cached"])
        p.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("gen,prec", [(0, 0), (1, 1)])
def test_row_group_on_two_processes_over_the_library(mf, gen, prec):
    """Two processes, each with its row-slice plan of the library (one with a
    partial cache of the pairs its rows touch), drive rowgroup.propagate with
    a gloo all-gather of host copies of the slices: both end with the
    oracle's exp(-i dt H) psi."""
    import torch.multiprocessing as tmp
    D, nvec = (1000, 2) if gen == 0 else (3000, 1)
    form = O.FORM_FP64 if prec == 0 else O.FORM_FP32
    op = O.make_op(gen, D, seed=6, form=form)
    if gen == 0:
        bounds = _padded_bounds(O.make_op(gen, D, seed=6))
        dt = 0.8
    else:
        dx = 2 * W.dvr_default_L(D) / (D - 1)
        bounds = None  # analytic on every rank
        emin, emax = 0.0, np.pi ** 2 / (2 * dx * dx) + 0.5 * W.dvr_default_L(D) ** 2
        dt = 2e-3
    psi = W.random_state(D, nvec, seed=8).reshape(D, nvec)
    world, port = 2, _free_port()
    case = (gen, prec, D, nvec, dt, bounds, psi)
    with tmp.get_context("spawn").Manager() as m:
        out = m.dict()
        tmp.spawn(_rank_main, args=(world, port, case, out), nprocs=world, join=True)
        res = dict(out)
    emin, emax = bounds if bounds is not None else (emin, emax)
    c, R = 0.5 * (emax + emin), 0.5 * (emax - emin)
    nt = O.cheb_terms(R * dt, 1e-13)
    ref = O.cheb_step(op, psi, dt, c, R, nt)
    tol = 1e-11 if prec == 0 else 2e-5 * np.max(np.abs(ref))
    for r in (0, 1):
        assert np.max(np.abs(res[r][2] - ref)) < tol
    assert res[1][3] > 0  # the second rank's slice cached its pairs


def test_slice_plans_refuse_what_they_cannot_do(mf):
    D = 1000
    x = torch.zeros((D, 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(mf.MFError):
        mf.Plan(D, 0, precision=0, row_begin=100, row_end=500)    # not a tile boundary
    with pytest.raises(mf.MFError):
        mf.Plan(D, 0, precision=2, row_begin=0, row_end=512)      # BF16X2 has no slice form
    p = mf.Plan(D, 0, precision=0, row_begin=0, row_end=512)
    with pytest.raises(mf.MFError):
        p.cheb_propagate(x, 1, 0.1, 4)                            # row groups use the rows calls
    with pytest.raises(mf.MFError):
        p.rows_cheb_begin(0.1)                                    # Philox slice without bounds
    p.close()
