"""Slab decomposition of one 3D transform over G processes / GPUs (the paper's slab scheme,
Sec. 2.2.1, with the exchange of Sec. 4.1 steps 2-4 as one all-to-all).

Layout.  The global grid (nx, ny, nz) is C-ordered, z contiguous.  Process r holds the
x-slab ``X_r = grid[r*nx/G : (r+1)*nx/G]`` (shape (nx/G, ny, nz)) before a forward
transform and the y-slab ``Y_r = spectrum[:, r*ny/G : (r+1)*ny/G]`` (shape (nx, ny/G, nz))
after it; the backward transform goes from y-slabs back to x-slabs, so forward then
backward returns every process its own slab times N.

Forward on process r:
  1. the z and y 1D transforms of its x-slab (``croft_exec_axes``, axes z|y), in place;
  2. pack: the slab viewed as [nx/G][G][ny/G * nz] becomes [G][nx/G][ny/G * nz]
     (``croft_transpose_blocks``): block s is what process s needs;
  3. one all-to-all with equal splits (``torch.distributed.all_to_all_single``; NCCL between
     GPUs): process r receives block r of every process s, in s order, which is exactly the
     C-ordered y-slab (nx, ny/G, nz) with x = s*nx/G + local x;
  4. the x 1D transforms of the y-slab (``croft_exec_axes``, axis x).
Backward on process r: the x transforms of its y-slab; the all-to-all (the y-slab already
is [G][nx/G][ny/G][nz], block s for process s); unpack [G][nx/G][ny/G*nz] ->
[nx/G][G][ny/G*nz] = the x-slab; the y and z transforms.

Every transform and copy runs in libcroft (its kernels and copy-engine copies); the
exchange is the one collective of the path.  `ops` replaces the libcroft steps (the CPU
tests drive the same partition and exchange schedule with a reference implementation of
the local steps); `exchange` replaces the all-to-all.
"""

from __future__ import annotations

AXIS_X, AXIS_Y, AXIS_Z = 1, 2, 4  # croft_exec_axes bit masks
FORWARD, BACKWARD = -1, +1


def slab_shapes(shape, world: int):
    """(x-slab shape, y-slab shape) of a grid split over `world` processes; ValueError if it does not split."""
    nx, ny, nz = (int(v) for v in shape)
    if world < 1 or nx % world or ny % world:
        raise ValueError(f"slab decomposition needs nx and ny divisible by the process count ({shape}, {world})")
    return (nx // world, ny, nz), (nx, ny // world, nz)


class CroftSlabOps:
    """The local steps on the GPU: libcroft plans of the two slab shapes and its block transpose."""

    def __init__(self, shape_x, shape_y, dtype):
        from . import croft
        self.croft = croft
        self.plan_x = croft.Plan(*shape_x, dtype=dtype)  # z and y passes of the x-slab
        self.plan_y = croft.Plan(*shape_y, dtype=dtype)  # x pass of the y-slab
        self.elem_bytes = 16 if dtype == croft.CROFT_C2C_F64 else 8

    def axes(self, which: str, inp, out, axes: int, direction: int, stream=None):
        plan = self.plan_x if which == "x" else self.plan_y
        self.croft.croft_exec_axes(plan.handle, inp, out, axes, direction, stream)

    def transpose(self, inp, out, d0: int, d1: int, inner: int, stream=None):
        self.croft.croft_transpose_blocks(inp, out, d0, d1, inner * self.elem_bytes, stream)

    def empty(self, like, n: int):
        import torch
        return torch.empty(n, dtype=like.dtype, device=like.device)

    def close(self):
        self.plan_x.close()
        self.plan_y.close()


def _all_to_all(send, recv, group=None):
    import torch
    import torch.distributed as dist
    if send.is_complex():
        send, recv = torch.view_as_real(send), torch.view_as_real(recv)
    dist.all_to_all_single(recv, send, group=group)


class SlabFFT:
    """One (nx, ny, nz) transform distributed in slabs over the processes of `group`."""

    def __init__(self, shape, world: int = None, rank: int = None, group=None, dtype=None, ops=None,
                 exchange=None):
        if world is None or rank is None:
            import torch.distributed as dist
            world = dist.get_world_size(group) if world is None else world
            rank = dist.get_rank(group) if rank is None else rank
        self.shape = tuple(int(v) for v in shape)
        self.world, self.rank, self.group = int(world), int(rank), group
        self.shape_x, self.shape_y = slab_shapes(self.shape, self.world)
        if ops is None:
            from . import croft
            ops = CroftSlabOps(self.shape_x, self.shape_y, croft.CROFT_C2C_F32 if dtype is None else dtype)
        self.ops = ops
        self.exchange = exchange or (lambda send, recv: _all_to_all(send, recv, self.group))
        nxl, ny, nz = self.shape_x
        self.n_local = nxl * ny * nz
        self.block = nxl * (ny // self.world) * nz  # elements sent to each process
        self._bufs = None

    def buffers(self, like):
        """(send, recv): the exchange buffers, N/G elements each (allocated on first use)."""
        if self._bufs is None:
            self._bufs = (self.ops.empty(like, self.n_local), self.ops.empty(like, self.n_local))
        return self._bufs

    # Each direction is two local stages around the exchange, so that the ranks of a job can
    # also be driven one stage at a time (the single-GPU test emulates G ranks this way).
    def forward_send(self, x_slab, stream=None, work=None):
        """Forward stage 1: z and y transforms of the x-slab (into `work`, default in place), packed
        for the exchange."""
        nxl, ny, nz = self.shape_x
        G = self.world
        send, _ = self.buffers(x_slab)
        work = x_slab if work is None else work
        self.ops.axes("x", x_slab, work, AXIS_Z | AXIS_Y, FORWARD, stream)
        self.ops.transpose(work, send, nxl, G, (ny // G) * nz, stream)  # [nxl][G][b] -> [G][nxl][b]
        return send

    def forward_finish(self, recv, out, stream=None):
        """Forward stage 2: the received blocks form the y-slab; its x transforms."""
        self.ops.axes("y", recv, out, AXIS_X, FORWARD, stream)
        return out

    def forward(self, x_slab, out, stream=None, work=None):
        """x-slab (nx/G, ny, nz) -> y-slab (nx, ny/G, nz) of Eq. (1).  `x_slab` is overwritten unless a
        separate `work` slab is given."""
        send = self.forward_send(x_slab, stream, work)
        recv = self.buffers(x_slab)[1]
        self.exchange(send, recv)
        return self.forward_finish(recv, out, stream)

    def backward_send(self, y_slab, stream=None, work=None):
        """Backward stage 1: x transforms of the y-slab (into `work`, default in place); block s is
        its x range s."""
        work = y_slab if work is None else work
        self.ops.axes("y", y_slab, work, AXIS_X, BACKWARD, stream)
        return work.reshape(-1)

    def backward_finish(self, recv, out, stream=None):
        """Backward stage 2: unpack the received blocks into the x-slab; its y and z transforms."""
        nxl, ny, nz = self.shape_x
        G = self.world
        self.ops.transpose(recv, out, G, nxl, (ny // G) * nz, stream)  # [G][nxl][b] -> [nxl][G][b]
        self.ops.axes("x", out, out, AXIS_Z | AXIS_Y, BACKWARD, stream)
        return out

    def backward(self, y_slab, out, stream=None, work=None):
        """y-slab (nx, ny/G, nz) -> x-slab (nx/G, ny, nz) of Eq. (2), unnormalised.  `y_slab` is
        overwritten unless a separate `work` slab is given."""
        send = self.backward_send(y_slab, stream, work)
        recv = self.buffers(y_slab)[1]
        self.exchange(send, recv)
        return self.backward_finish(recv, out, stream)

    def close(self):
        if hasattr(self.ops, "close"):
            self.ops.close()


def partition_grids(dims, world: int):
    """Split a batch of independent grids over `world` processes (no exchange: each grid is a
    unit of its own).  Longest processing time first on the nominal cost N log2 N: grids in
    decreasing cost, each to the currently least loaded process (ties to the lower rank).
    Returns one list of grid indices per process, each in the batch's order."""
    import math
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = []
    for i, d in enumerate(dims):
        n = int(d[0]) * int(d[1]) * int(d[2])
        cost.append((n * math.log2(n) if n > 1 else 0.0, i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for c, i in sorted(cost, key=lambda t: (-t[0], t[1])):
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += c
    return [sorted(p) for p in parts]
