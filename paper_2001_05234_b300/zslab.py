"""One Poisson solve split over ranks by z-slabs (one process per GPU).

Rank r of P owns the z-planes z0 .. z1-1 of the whole problem, all of x and y.  Its x-y transforms
are local (a plan of the slab's shape); the tridiagonal systems along z (Eq. poi_reduced) cross the
slabs through one exchange: each rank's elimination pass (cans_zslab_eliminate) leaves 10 numbers per
(x, y) column, every rank gathers all of them (an all-gather, NCCL between GPUs), and the finish pass
(cans_zslab_finish) solves the P-unknown reduced system of the slabs' last rows and back-substitutes
its own slab.  This module only places data and calls the library and the collective: every
arithmetic step runs in the library's kernels.  FP64 plans, wall-bounded z.
"""
from __future__ import annotations

from . import (CANS_BC_NN, CANS_FP64, _check, _stream_ptr, cans_opts_default, cans_plan_destroy, cans_poisson_plan,
               cans_transform_xy, cans_zslab_create, cans_zslab_destroy, cans_zslab_eliminate, cans_zslab_finish,
               cans_zslab_sizes)


def slab_ranges(nz: int, nranks: int):
    """Contiguous z-slabs [z0, z1) for each rank: sizes differ by at most one plane, the larger ones
    first; every rank gets at least one plane."""
    if nranks < 1 or nz < nranks:
        raise ValueError(f"{nz} planes cannot be split over {nranks} ranks")
    base, extra = divmod(nz, nranks)
    out, z = [], 0
    for r in range(nranks):
        h = base + (1 if r < extra else 0)
        out.append((z, z + h))
        z += h
    return out


def gather_exchange(group=None):
    """The exchange of a distributed run: torch.distributed all-gathers of every rank's interface
    numbers (equal sizes) and singular-column pieces (uneven: padded to the largest slab, then cut)."""
    import torch
    import torch.distributed as dist

    def exchange(iface, col00, slabs):
        world = dist.get_world_size(group)
        parts = [torch.empty_like(iface) for _ in range(world)]
        dist.all_gather(parts, iface, group=group)
        hmax = max(z1 - z0 for z0, z1 in slabs)
        pad = torch.zeros(hmax, dtype=col00.dtype, device=col00.device)
        pad[: col00.numel()] = col00
        cols = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(cols, pad, group=group)
        col_all = torch.cat([cols[r][: z1 - z0] for r, (z0, z1) in enumerate(slabs)])
        return torch.cat(parts), col_all

    return exchange


class ZSlabSolver:
    """Rank `rank`'s part of a solve of L_h p = f split over `nranks` z-slabs.  f and p are the rank's
    slabs: float64 CUDA tensors of shape (z1 - z0, Ny, Nx)."""

    def __init__(self, n, bc, length_xy, dzf, nranks: int, rank: int):
        import torch

        self.n = tuple(int(v) for v in n)
        self.nranks, self.rank = int(nranks), int(rank)
        self.slabs = slab_ranges(self.n[2], self.nranks)
        self.z0, self.z1 = self.slabs[self.rank]
        o = cans_opts_default()
        o.prec = CANS_FP64
        _, self.plan = cans_poisson_plan(self.n, length_xy, tuple(bc), dzf, o)
        # the slab's x-y transforms (their tables do not depend on z)
        _, self.xy_plan = cans_poisson_plan((self.n[0], self.n[1], self.z1 - self.z0), length_xy,
                                            (bc[0], bc[1], CANS_BC_NN), None, o)
        self.slab = cans_zslab_create(self.plan, self.z0, self.z1)
        ws, nif, ncol = cans_zslab_sizes(self.slab)
        self._ws_buf = torch.empty(ws + 256, dtype=torch.uint8, device="cuda")
        self._ws = self._ws_buf.data_ptr() + (-self._ws_buf.data_ptr()) % 256
        self.iface = torch.empty(nif, dtype=torch.float64, device="cuda")
        self.col00 = torch.empty(ncol, dtype=torch.float64, device="cuda")

    @property
    def shape(self):
        return (self.z1 - self.z0, self.n[1], self.n[0])

    def eliminate(self, f, out, stream=None):
        """x-y transforms of the slab and the slab's elimination pass; returns the numbers to exchange."""
        import torch

        assert f.dtype == torch.float64 and f.is_cuda and tuple(f.shape) == self.shape
        out.copy_(f)
        sp = _stream_ptr(stream)
        _check(cans_transform_xy(self.xy_plan, out.data_ptr(), 1, sp), "cans_transform_xy")
        _check(cans_zslab_eliminate(self.slab, out.data_ptr(), self.iface.data_ptr(), self.col00.data_ptr(), self._ws,
                                    sp), "cans_zslab_eliminate")
        return self.iface, self.col00

    def finish(self, out, iface_all, col00_all, stream=None):
        """The reduced system, the slab's back substitution and the inverse x-y transforms."""
        sp = _stream_ptr(stream)
        scale = 1.0 / (self.n[0] * self.n[1])
        _check(cans_zslab_finish(self.slab, out.data_ptr(), iface_all.data_ptr(), col00_all.data_ptr(), self.nranks,
                                 self.rank, scale, self._ws, sp), "cans_zslab_finish")
        _check(cans_transform_xy(self.xy_plan, out.data_ptr(), -1, sp), "cans_transform_xy")
        return out

    def solve(self, f, out=None, exchange=None, stream=None):
        """The whole solve on this rank: eliminate, exchange (default: torch.distributed all-gathers),
        finish."""
        import torch

        out = torch.empty_like(f) if out is None else out
        iface, col00 = self.eliminate(f, out, stream)
        iface_all, col00_all = (exchange or gather_exchange())(iface, col00, self.slabs)
        return self.finish(out, iface_all, col00_all, stream)

    def close(self):
        for name in ("slab",):
            if getattr(self, name, None):
                cans_zslab_destroy(getattr(self, name))
                setattr(self, name, None)
        for name in ("plan", "xy_plan"):
            if getattr(self, name, None):
                cans_plan_destroy(getattr(self, name))
                setattr(self, name, None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["slab_ranges", "gather_exchange", "ZSlabSolver"]
