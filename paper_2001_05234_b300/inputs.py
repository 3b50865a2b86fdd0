"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module only draws random numbers and builds the synthetic workloads (grids, right-hand sides,
initial velocity fields).  It holds none of the solver's arithmetic, so the CUDA path and the CPU
oracle can both consume its output without sharing any method code.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds.  A
uniform double takes the top 53 bits; normals use the Box-Muller transform.  The host (numpy) and
device (torch) generators produce the same 64-bit words.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

BC_P, BC_NN, BC_DD = 0, 1, 2
BC_ND, BC_DN = 3, 4  # z only: Neumann low / Dirichlet high wall, and the reverse
BC_NAMES = {BC_P: "P", BC_NN: "NN", BC_DD: "DD"}

SEED_BASE = 2001052340  # config c draws from seed SEED_BASE + c


def _stream_seed(seed: int, stream: int) -> int:
    return (seed + 0x632BE59BD9B4E019 * stream) & MASK64


# ----------------------------------------------------------------------------------------------
# host (numpy) generator
# ----------------------------------------------------------------------------------------------
def splitmix64(seed: int, count: int, offset: int = 0, stream: int = 0) -> np.ndarray:
    """Words offset .. offset+count-1 of the SplitMix64 sequence started at ``seed`` (uint64)."""
    s = np.uint64(_stream_seed(seed, stream))
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = s + idx * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, shape, lo: float = 0.0, hi: float = 1.0, stream: int = 0) -> np.ndarray:
    n = int(np.prod(shape))
    u = (splitmix64(seed, n, stream=stream) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return (lo + (hi - lo) * u).reshape(shape)


def normal(seed: int, shape, stream: int = 0) -> np.ndarray:
    n = int(np.prod(shape))
    u1 = 1.0 - uniform(seed, (n,), stream=2 * stream + 100)  # (0, 1]
    u2 = uniform(seed, (n,), stream=2 * stream + 101)
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).reshape(shape)


def randint(seed: int, count: int, lo: int, hi: int, stream: int = 0) -> np.ndarray:
    """Integers uniform on lo..hi inclusive (modulo draw; bias < 2^-50 for the ranges used here)."""
    w = splitmix64(seed, count, stream=stream)
    return (lo + (w % np.uint64(hi - lo + 1)).astype(np.int64)).astype(np.int64)


# ----------------------------------------------------------------------------------------------
# device (torch) generator: same words as the host one
# ----------------------------------------------------------------------------------------------
def _signed(v: int) -> int:
    v &= MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def splitmix64_torch(seed: int, count: int, device, offset: int = 0, stream: int = 0):
    import torch

    s = _signed(_stream_seed(seed, stream))
    idx = torch.arange(offset + 1, offset + count + 1, dtype=torch.int64, device=device)
    z = idx * _signed(GAMMA) + s

    def lsr(x, k):
        return (x >> k) & ((1 << (64 - k)) - 1)

    z = (z ^ lsr(z, 30)) * _signed(M1)
    z = (z ^ lsr(z, 27)) * _signed(M2)
    return z ^ lsr(z, 31)


def uniform_torch(seed: int, count: int, device, lo=0.0, hi=1.0, stream: int = 0, chunk: int = 1 << 26):
    import torch

    out = torch.empty(count, dtype=torch.float64, device=device)
    for o in range(0, count, chunk):
        c = min(chunk, count - o)
        w = splitmix64_torch(seed, c, device, offset=o, stream=stream)
        u = ((w >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
        out[o:o + c] = lo + (hi - lo) * u
    return out


def normal_torch(seed: int, count: int, device, stream: int = 0, chunk: int = 1 << 26):
    import torch

    out = torch.empty(count, dtype=torch.float64, device=device)
    for o in range(0, count, chunk):
        c = min(chunk, count - o)
        w1 = splitmix64_torch(seed, c, device, offset=o, stream=2 * stream + 100)
        w2 = splitmix64_torch(seed, c, device, offset=o, stream=2 * stream + 101)
        u1 = 1.0 - ((w1 >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
        u2 = ((w2 >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
        out[o:o + c] = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
    return out


# ----------------------------------------------------------------------------------------------
# grids
# ----------------------------------------------------------------------------------------------
def tanh_dzf(nz: int, alpha: float, lz: float = 1.0) -> np.ndarray:
    """Cell widths of the wall-clustered grid with faces z_k = lz/2 (1 + tanh(alpha (2k/nz - 1))/tanh(alpha)),
    k = 0..nz (two-sided tanh clustering of the Validation section, written for faces)."""
    k = np.arange(nz + 1, dtype=np.float64)
    zf = 0.5 * lz * (1.0 + np.tanh(alpha * (2.0 * k / nz - 1.0)) / np.tanh(alpha))
    zf[0], zf[-1] = 0.0, lz
    return np.diff(zf)


def uniform_dzf(nz: int, lz: float = 1.0) -> np.ndarray:
    return np.full(nz, lz / nz)


def z_centres(dzf: np.ndarray) -> np.ndarray:
    zf = np.concatenate([[0.0], np.cumsum(dzf)])
    return 0.5 * (zf[:-1] + zf[1:])


def weighted_mean_removed(f: np.ndarray, dzf: np.ndarray) -> np.ndarray:
    """Subtract the cell-volume-weighted mean (x, y uniform; z weights dzf)."""
    w = dzf / dzf.sum()
    m = float((f.mean(axis=(1, 2)) * w).sum())
    return f - m


def seven_point_average(f: np.ndarray, bc) -> np.ndarray:
    """One pass of (centre + 6 neighbours)/7; periodic directions wrap, wall directions clamp the index."""
    out = f.copy()
    for axis, b in zip((2, 1, 0), bc):  # array axes are (z, y, x); bc is (x, y, z)
        n = f.shape[axis]
        if b == BC_P:
            out += np.roll(f, 1, axis=axis) + np.roll(f, -1, axis=axis)
        else:
            idx_m = np.clip(np.arange(n) - 1, 0, n - 1)
            idx_p = np.clip(np.arange(n) + 1, 0, n - 1)
            out += np.take(f, idx_m, axis=axis) + np.take(f, idx_p, axis=axis)
    return out / 7.0


# ----------------------------------------------------------------------------------------------
# Poisson workloads
# ----------------------------------------------------------------------------------------------
@dataclass
class PoissonCase:
    name: str
    n: tuple  # (nx, ny, nz)
    bc: tuple  # (bx, by, bz)
    length_xy: tuple
    dzf: np.ndarray
    seed: int
    rhs_kind: str  # "uniform", "gauss7", "modes"
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    @property
    def points(self):
        return self.n[0] * self.n[1] * self.n[2]


def case_uniform32(n=(32, 32, 32), seed=SEED_BASE + 1) -> PoissonCase:
    """32^3, unit box, x/y periodic, z Neumann-Neumann, uniform grid; f ~ U[-1,1] minus its mean."""
    return PoissonCase("uniform32", tuple(n), (BC_P, BC_P, BC_NN), (1.0, 1.0), uniform_dzf(n[2]), seed, "uniform")


def case_channel(n=(1024, 512, 256), alpha=1.8, seed=SEED_BASE + 2) -> PoissonCase:
    """Channel-type problem: x periodic, y Dirichlet-Dirichlet, z Neumann-Neumann on tanh faces."""
    return PoissonCase("channel", tuple(n), (BC_P, BC_DD, BC_NN), (1.0, 1.0), tanh_dzf(n[2], alpha), seed, "gauss7")


def case_modes(n=(1024, 1024, 512), alpha=1.8, seed=SEED_BASE + 3, n_modes=64, noise=1e-3) -> PoissonCase:
    """x, y periodic, z Neumann on tanh faces; f = sum of random separable Fourier modes + N(0, noise)."""
    return PoissonCase("modes", tuple(n), (BC_P, BC_P, BC_NN), (1.0, 1.0), tanh_dzf(n[2], alpha), seed, "modes",
                       {"n_modes": n_modes, "noise": noise})


def _mode_factors(case: PoissonCase):
    """1-D factors of the separable Fourier-mode RHS (host, FP64): cx[m, i], cy[m, j], cz[m, k], a[m]."""
    nx, ny, nz = case.n
    nm = case.extra["n_modes"]
    kx = randint(case.seed, nm, 0, nx // 2 - 1, stream=1)
    ky = randint(case.seed, nm, 0, ny // 2 - 1, stream=2)
    kz = randint(case.seed, nm, 0, nz - 1, stream=3)
    amp = uniform(case.seed, (nm,), -1.0, 1.0, stream=4)
    phx = uniform(case.seed, (nm,), 0.0, 2 * np.pi, stream=5)
    phy = uniform(case.seed, (nm,), 0.0, 2 * np.pi, stream=6)
    lx, ly = case.length_xy
    xc = (np.arange(nx) + 0.5) * lx / nx
    yc = (np.arange(ny) + 0.5) * ly / ny
    zc = z_centres(case.dzf)
    lz = float(case.dzf.sum())
    cx = np.cos(2 * np.pi * kx[:, None] * xc[None, :] / lx + phx[:, None])
    cy = np.cos(2 * np.pi * ky[:, None] * yc[None, :] / ly + phy[:, None])
    cz = np.cos(np.pi * kz[:, None] * zc[None, :] / lz)
    return cx, cy, cz, amp


def rhs_host(case: PoissonCase) -> np.ndarray:
    """The case's right-hand side as a host array of shape (nz, ny, nx), compatible (zero weighted mean)."""
    shape = case.shape
    if case.rhs_kind == "uniform":
        f = uniform(case.seed, shape, -1.0, 1.0)
    elif case.rhs_kind == "gauss7":
        f = seven_point_average(normal(case.seed, shape), case.bc)
    elif case.rhs_kind == "modes":
        cx, cy, cz, amp = _mode_factors(case)
        f = np.einsum("m,mk,mj,mi->kji", amp, cz, cy, cx, optimize=True)
        f = f + case.extra["noise"] * normal(case.seed, shape, stream=7)
    else:
        raise ValueError(case.rhs_kind)
    return weighted_mean_removed(f, case.dzf)


def rhs_device(case: PoissonCase, device):
    """Same recipe generated on a torch device (used for the large cases)."""
    import torch

    nz, ny, nx = case.shape
    n = nx * ny * nz
    w = torch.tensor(case.dzf / case.dzf.sum(), dtype=torch.float64, device=device)
    if case.rhs_kind == "uniform":
        f = uniform_torch(case.seed, n, device, -1.0, 1.0).view(nz, ny, nx)
    elif case.rhs_kind == "gauss7":
        g = normal_torch(case.seed, n, device).view(nz, ny, nx)
        f = g.clone()
        for dim, b in zip((2, 1, 0), case.bc):
            if b == BC_P:
                f += torch.roll(g, 1, dims=dim) + torch.roll(g, -1, dims=dim)
            else:
                m = g.shape[dim]
                im = torch.clamp(torch.arange(m, device=device) - 1, 0, m - 1)
                ip = torch.clamp(torch.arange(m, device=device) + 1, 0, m - 1)
                f += torch.index_select(g, dim, im) + torch.index_select(g, dim, ip)
        del g
        f /= 7.0
    elif case.rhs_kind == "modes":
        cx, cy, cz, amp = _mode_factors(case)
        cx = torch.tensor(cx, device=device)
        czy = torch.tensor(np.einsum("m,mk,mj->kjm", amp, cz, cy), device=device).reshape(nz * ny, -1)
        f = (czy @ cx).view(nz, ny, nx)
        del czy
        f += case.extra["noise"] * normal_torch(case.seed, n, device, stream=7).view(nz, ny, nx)
    else:
        raise ValueError(case.rhs_kind)
    m = (f.mean(dim=(1, 2)) * w).sum()
    f -= m
    return f.contiguous()


def ensemble_cases(count=64, seed=SEED_BASE + 5, sizes=(32, 48, 64, 96, 128, 192)):
    """Uneven ensemble: every dimension from `sizes`, the boundary condition of every direction from
    {periodic, Neumann, Dirichlet}; a non-periodic z is uniform (probability 1/2) or tanh-stretched
    with alpha ~ U[1.0, 2.2]; unit box; f ~ U[-1, 1] (made compatible by rhs_host)."""
    cases = []
    dims = randint(seed, 3 * count, 0, len(sizes) - 1, stream=21).reshape(count, 3)
    bcs = randint(seed, 3 * count, 0, 2, stream=22).reshape(count, 3)
    coin = uniform(seed, (count,), stream=23)
    alphas = uniform(seed, (count,), 1.0, 2.2, stream=24)
    for q in range(count):
        n = tuple(int(sizes[d]) for d in dims[q])
        bc = tuple(int(b) for b in bcs[q])
        if bc[2] == BC_P or coin[q] < 0.5:
            dzf = uniform_dzf(n[2])
        else:
            dzf = tanh_dzf(n[2], float(alphas[q]))
        cases.append(PoissonCase(f"ensemble{q}", n, bc, (1.0, 1.0), dzf, seed * 1000 + q, "uniform"))
    return cases
