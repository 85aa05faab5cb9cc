"""Row-distributed Chebyshev propagation across ranks (the row-parallel mode
of Sec. IV.H): rank j holds a plan for its rows R_j (``row_begin``,
``row_end``; its cache holds the blocks those rows touch) and the whole
vector.  Every recurrence term is the library's slice update on each rank,
then an all-gather of the new slices (the one collective of the path, as in
Sec. IV.H: linear in D against the quadratic product).

The driver only orders library calls and the collective; all arithmetic runs
in the library's kernels.
"""


def propagate(plan, psi_full, nvec, dt, allgather, order=0):
    """One step psi <- exp(-i dt H) psi.

    plan       -- this rank's Plan, created with row_begin / row_end
    psi_full   -- device complex128 tensor [D][nvec], identical on every rank
    allgather  -- callable: this rank's [rows][nvec] slice -> the [D][nvec]
                  concatenation of every rank's slice in row order
    Returns the new psi on all rows (gathered).
    """
    import torch
    rows = plan.row_end - plan.row_begin
    nt = plan.rows_cheb_begin(dt, order)
    acc = torch.empty((rows, nvec), dtype=torch.complex128, device=psi_full.device)
    q_prev = torch.zeros_like(acc)
    q_next = torch.empty_like(acc)
    plan.rows_cheb_init(psi_full, acc, nvec)
    q_full = psi_full
    for j in range(1, nt):
        plan.rows_cheb_term(j, q_full, q_prev, q_next, acc, nvec)
        q_full = allgather(q_next)
    out = torch.empty_like(acc)
    plan.rows_cheb_final(acc, out, nvec, dt)
    return allgather(out)


def slices(D, world, tile=128):
    """Row slices [begin, end) for world ranks: whole 128-row tiles, the
    remainder spread over the first ranks, the last slice ending at D."""
    ntile = -(-D // tile)
    base, extra = divmod(ntile, world)
    out, t = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((t * tile, min(D, (t + n) * tile)))
        t += n
    return out


def dist_allgather(group=None, host=False):
    """An allgather for torch.distributed (NCCL on GPUs, gloo on CPU) that
    accepts slices of unequal length (padded to the longest, then trimmed).
    The slice lengths are fixed by the plans, so they are exchanged once, on
    the first call, and again only if this rank's length changes.  host=True
    gathers host copies (for a CPU-only backend such as gloo driving device
    tensors) and returns the result on the input's device."""
    import torch
    import torch.distributed as dist

    known = {"local": None, "sizes": None}

    def gather(t):
        dev = t.device
        if host:
            t = t.cpu()
        world = dist.get_world_size(group)
        if known["local"] != t.shape[0]:
            n = torch.tensor([t.shape[0]], device=t.device)
            sizes = [torch.zeros_like(n) for _ in range(world)]
            dist.all_gather(sizes, n, group=group)
            known["local"] = t.shape[0]
            known["sizes"] = [int(s.item()) for s in sizes]
        sizes = known["sizes"]
        m = max(sizes)
        pad = torch.zeros((m,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
        pad[: t.shape[0]] = t
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad, group=group)
        out = torch.cat([p[:s] for p, s in zip(parts, sizes)], dim=0)
        return out.to(dev) if host else out

    return gather
