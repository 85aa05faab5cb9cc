"""The N > 1 path of the benchmark on CPU: two gloo ranks run the same
host-side logic the GPU ranks run (independent task per rank, max-over-ranks
job time, whole-job value), with no data-path collective."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = 1.0 + rank             # rank 1 is the slower one
        t_job = bench.job_seconds(t_local, world)
        value = bench.job_value(world, 10, 1e9, t_job)
        out[rank] = (bench.rank_task(rank), t_job, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_job_time():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] != res[1][0]                     # independent problems
    assert res[0][1] == res[1][1] == 2.0              # slowest rank's time
    assert res[0][2] == res[1][2] == 2 * 10 * 1e9 / 2.0


class _OracleSlicePlan:
    """The row-slice calls of the library (mf_rows_cheb_*) restated on the
    oracle for a CPU run: y = H q on rows [r0, r1), the slice recurrence."""

    def __init__(self, op, r0, r1, c, R):
        self.op, self.row_begin, self.row_end, self.c, self.R = op, r0, r1, c, R

    def rows_cheb_begin(self, dt, order):
        from oracle import oracle as O
        self.J = O.bessel_j(self.R * dt, order + 8)
        return order

    def rows_cheb_init(self, psi_full, acc, nvec):
        acc[:] = self.J[0] * psi_full[self.row_begin:self.row_end]

    def rows_cheb_term(self, j, q_full, q_prev, q_next, acc, nvec):
        import numpy as np
        from oracle import oracle as O
        rows = np.arange(self.row_begin, self.row_end)
        y = torch.from_numpy(O.apply_rows(self.op, q_full.numpy(), rows))
        q = q_full[self.row_begin:self.row_end]
        t = (y - self.c * q) / self.R
        qn = t if j == 1 else 2 * t - q_prev
        q_prev[:] = q
        q_next[:] = qn
        acc += 2 * (-1j) ** j * self.J[j] * qn

    def rows_cheb_final(self, acc, out, nvec, dt):
        import numpy as np
        out[:] = np.exp(-1j * self.c * dt) * acc


def _row_worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2606_31598_gb300 import rowgroup
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        D, dt, nt, c, R = 300, 0.6, 24, 0.0, 2.3
        op = O.make_op(O.GEN_PHILOX_GUE, D, seed=7)
        r0, r1 = rowgroup.slices(D, world)[rank]
        plan = _OracleSlicePlan(op, r0, r1, c, R)
        rng = np.random.default_rng(1)
        psi = rng.standard_normal((D, 2)) + 1j * rng.standard_normal((D, 2))
        res = rowgroup.propagate(plan, torch.from_numpy(psi), 2, dt, rowgroup.dist_allgather(), order=nt)
        out[rank] = (r0, r1, res.numpy())
    finally:
        dist.destroy_process_group()


def test_row_group_propagation_on_two_gloo_ranks():
    """Two ranks own rows [0, 256) and [256, 300) (unequal slices); the
    driver's slice terms and all-gathers give the single-process step."""
    import numpy as np
    import torch.multiprocessing as mp
    from oracle import oracle as O
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_row_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert (res[0][0], res[0][1], res[1][0], res[1][1]) == (0, 256, 256, 300)
    D = 300
    op = O.make_op(O.GEN_PHILOX_GUE, D, seed=7)
    rng = np.random.default_rng(1)
    psi = rng.standard_normal((D, 2)) + 1j * rng.standard_normal((D, 2))
    ref = O.cheb_step(op, psi, 0.6, 0.0, 2.3, 24)
    for r in (0, 1):
        assert np.max(np.abs(res[r][2] - ref)) < 1e-12
