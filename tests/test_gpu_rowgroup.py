"""Row-distributed plans (row-parallel mode, Sec. IV.H) on one GPU: plans for
row slices apply H[rows, :] to the whole vector and cache only the pairs
their rows touch; several slice plans stepped in lockstep, with the gathers
emulated by concatenation, give the single plan's Chebyshev step.

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


def test_lockstep_row_group_step_matches_one_plan(mf):
    """Two slice plans stepped term by term (gather = concatenation) against
    one plan's exp(-i dt H) psi; the Philox slices get the same bounds."""
    from paper_2606_31598_gb300 import rowgroup
    D, nvec, dt = 1000, 2, 0.8
    full = mf.Plan(D, 0, seed=6, precision=0, cheb_tol=1e-13)
    emin, emax = full.bounds()
    psi = W.random_state(D, nvec, seed=5).reshape(D, nvec)
    ref_d = torch.from_numpy(psi.copy()).cuda()
    full.cheb_propagate(ref_d, nvec, dt, 0)
    nt_full = full.cheb_terms(dt)
    plans = []
    for r0, r1 in rowgroup.slices(D, 2):
        p = mf.Plan(D, 0, seed=6, precision=0, cheb_tol=1e-13, row_begin=r0, row_end=r1)
        p.set_bounds(emin, emax)
        plans.append(p)
    nts = [p.rows_cheb_begin(dt) for p in plans]
    assert nts[0] == nts[1] == nt_full
    psi_d = torch.from_numpy(psi).cuda()
    st = []
    for p in plans:
        rows = p.row_end - p.row_begin
        acc = torch.empty((rows, nvec), dtype=torch.complex128, device="cuda")
        p.rows_cheb_init(psi_d, acc, nvec)
        st.append([acc, torch.zeros_like(acc), torch.empty_like(acc)])
    q_full = psi_d
    for j in range(1, nt_full):
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
    assert np.max(np.abs(got - ref_d.cpu().numpy())) < 1e-11


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
