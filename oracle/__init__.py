"""CPU oracle for the pressure-Poisson hot path -- TEST INFRASTRUCTURE ONLY.

A plain FP64 (also long double / __float128) C++ implementation of the exact solution of the
7-point staggered Poisson equation (eq. poi) reached by eigenfunction expansion in x and y and a
Thomas solve along z (eq. poi_reduced), with dense closed-form eigenbases instead of FFTs.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
package.  The product path never does: it shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.cpp")

BC_P, BC_NN, BC_DD = 0, 1, 2
BC_ND, BC_DN = 3, 4  # z only: Neumann low / Dirichlet high wall, and the reverse


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (OpenMP, libquadmath).  Returns the path."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-o", _SO + ".tmp", _SRC, "-lquadmath"]
        subprocess.check_call(cmd)
        os.replace(_SO + ".tmp", _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_poisson_solve.argtypes = [ctypes.c_int, ip, dp, ip, dp, dp, dp, ctypes.c_int]
        L.oracle_apply_laplacian.argtypes = [ctypes.c_int, ip, dp, ip, dp, dp, dp, ctypes.c_int]
        L.oracle_eigenbasis.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        L.oracle_z_rows.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        L.oracle_thomas.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp]
        L.oracle_set_fault.argtypes = [ctypes.c_int]
        L.oracle_helmholtz_solve.argtypes = [ctypes.c_int, ip, dp, ip, dp, ctypes.c_double, ctypes.c_int, dp, dp,
                                             ctypes.c_int]
        L.oracle_apply_helmholtz.argtypes = [ctypes.c_int, ip, dp, ip, dp, ctypes.c_double, ctypes.c_int, dp, dp,
                                             ctypes.c_int]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _dz(n, dzf):
    if dzf is None:
        return np.full(n[2], 1.0 / n[2])
    dzf = np.ascontiguousarray(dzf, dtype=np.float64)
    assert dzf.shape == (n[2],)
    return dzf


def poisson_solve(f, bc, length_xy=(1.0, 1.0), dzf=None, prec=64, nthreads=0):
    """p with L_h p = f.  f has shape (nz, ny, nx) (x fastest).  Singular cases: zero-mean p."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    nz, ny, nx = f.shape
    n = np.array([nx, ny, nz], dtype=np.int32)
    b = np.array(bc, dtype=np.int32)
    L = np.array(length_xy, dtype=np.float64)
    dz = _dz(n, dzf)
    p = np.empty_like(f)
    rc = lib().oracle_poisson_solve(prec, _i(n), _d(L), _i(b), _d(dz), _d(f), _d(p), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_poisson_solve rejected its arguments (rc={rc})")
    return p


def apply_laplacian(p, bc, length_xy=(1.0, 1.0), dzf=None, prec=64, nthreads=0):
    """L_h p (eq. poi with a non-uniform z grid)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    nz, ny, nx = p.shape
    n = np.array([nx, ny, nz], dtype=np.int32)
    b = np.array(bc, dtype=np.int32)
    L = np.array(length_xy, dtype=np.float64)
    dz = _dz(n, dzf)
    out = np.empty_like(p)
    rc = lib().oracle_apply_laplacian(prec, _i(n), _d(L), _i(b), _d(dz), _d(p), _d(out), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_apply_laplacian rejected its arguments (rc={rc})")
    return out


def eigenbasis(bc, n):
    """(E, lam): orthonormal eigenvectors (columns) and unit-spacing eigenvalues of the 1-D operator."""
    E = np.empty((n, n))
    lam = np.empty(n)
    if lib().oracle_eigenbasis(int(bc), int(n), _d(E), _d(lam)) != 0:
        raise ValueError("bad eigenbasis arguments")
    return E, lam


def z_rows(bc_z, dzf):
    dzf = np.ascontiguousarray(dzf, dtype=np.float64)
    nz = dzf.shape[0]
    a, b, c = np.empty(nz), np.empty(nz), np.empty(nz)
    if lib().oracle_z_rows(int(bc_z), nz, _d(dzf), _d(a), _d(b), _d(c)) != 0:
        raise ValueError("bad z_rows arguments")
    return a, b, c


def thomas(a, b, c, d):
    a, b, c, d = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c, d))
    x = np.empty_like(d)
    lib().oracle_thomas(d.shape[0], _d(a), _d(b), _d(c), _d(d), _d(x))
    return x


def set_fault(mode: int) -> None:
    """Plant one deliberate mistake (mutation tests only); 0 restores the correct oracle."""
    lib().oracle_set_fault(int(mode))


def relative_residual(p, f, bc, length_xy=(1.0, 1.0), dzf=None, nthreads=0, shift=0.0, z_grid=0):
    if shift == 0.0 and z_grid == 0:
        r = apply_laplacian(p, bc, length_xy, dzf, nthreads=nthreads) - f
    else:
        r = apply_helmholtz(p, bc, length_xy, dzf, shift=shift, z_grid=z_grid, nthreads=nthreads) - f
    return float(np.linalg.norm(r) / np.linalg.norm(f))


# ---- Helmholtz form (Eq. up_id_2) and the face grid of a staggered w ------------------------------
def _helm_args(shape, bc, length_xy, dzf, z_grid):
    nu, ny, nx = shape
    ncell = nu + int(z_grid)
    n = np.array([nx, ny, ncell], dtype=np.int32)
    return n, np.array(bc, dtype=np.int32), np.array(length_xy, dtype=np.float64), _dz(n, dzf)


def helmholtz_solve(f, bc, length_xy=(1.0, 1.0), dzf=None, shift=0.0, z_grid=0, prec=64, nthreads=0):
    """p with (L_h + shift) p = f.  z_grid 0: f is (nz, ny, nx) on the cell centres of the nz dzf cells;
    z_grid 1: f is (nz - 1, ny, nx) on the interior z-faces (w = 0 on the wall faces; bc_z Dirichlet)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    n, b, L, dz = _helm_args(f.shape, bc, length_xy, dzf, z_grid)
    p = np.empty_like(f)
    rc = lib().oracle_helmholtz_solve(prec, _i(n), _d(L), _i(b), _d(dz), float(shift), int(z_grid), _d(f), _d(p),
                                      int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_helmholtz_solve rejected its arguments (rc={rc})")
    return p


def apply_helmholtz(p, bc, length_xy=(1.0, 1.0), dzf=None, shift=0.0, z_grid=0, prec=64, nthreads=0):
    """(L_h + shift) p on the grid of helmholtz_solve."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    n, b, L, dz = _helm_args(p.shape, bc, length_xy, dzf, z_grid)
    out = np.empty_like(p)
    rc = lib().oracle_apply_helmholtz(prec, _i(n), _d(L), _i(b), _d(dz), float(shift), int(z_grid), _d(p), _d(out),
                                      int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_apply_helmholtz rejected its arguments (rc={rc})")
    return out


# ---- fractional-step pieces (channel: x, y periodic, walls in z) --------------------------------
def _chan_args(shape, length_xy, dzf):
    nz, ny, nx = shape
    n = np.array([nx, ny, nz], dtype=np.int32)
    L = np.array(length_xy, dtype=np.float64)
    dz = _dz(n, dzf)
    return n, L, dz


def _bind_chan():
    L = lib()
    if getattr(L, "_chan_bound", False):
        return L
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    L.oracle_divergence.argtypes = [ip, dp, dp, dp, dp, dp, dp]
    L.oracle_gradient.argtypes = [ip, dp, dp, dp, dp, dp, dp]
    L.oracle_momentum_rhs.argtypes = [ip, dp, dp, ctypes.c_double, dp, dp, dp, dp, dp, dp]
    L.oracle_stable_dt.argtypes = [ip, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
    L.oracle_stable_dt.restype = ctypes.c_double
    L.oracle_project.argtypes = [ip, dp, dp, dp, dp, dp, dp, dp, dp, dp, ctypes.c_int]
    L.oracle_rk3_step.argtypes = [ip, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  dp, dp, dp, dp, dp, ctypes.c_int]
    L.oracle_rk3_step_implicit.argtypes = [ip, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_double, dp, dp, dp, dp, dp, ctypes.c_int]
    L.oracle_box_project.argtypes = [ip, ip, dp, dp, dp, dp, dp, ctypes.c_int]
    L.oracle_box_divergence.argtypes = [ip, ip, dp, dp, dp, dp, dp, dp]
    L.oracle_box_operators.argtypes = [ip, ip, ctypes.c_double, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
    L.oracle_box_rk3_step.argtypes = [ip, ip, ctypes.c_double, dp, dp, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_double, dp, dp, dp, dp, dp,
                                      ctypes.c_int]
    L._chan_bound = True
    return L


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def divergence(u, v, w, length_xy, dzf):
    """Cell-centred divergence of a face field (w is zero on both walls; w[-1] is the top wall)."""
    L = _bind_chan()
    u, v, w = _c(u), _c(v), _c(w)
    n, Lxy, dz = _chan_args(u.shape, length_xy, dzf)
    out = np.empty_like(u)
    L.oracle_divergence(_i(n), _d(Lxy), _d(dz), _d(u), _d(v), _d(w), _d(out))
    return out


def gradient(q, length_xy, dzf):
    L = _bind_chan()
    q = _c(q)
    n, Lxy, dz = _chan_args(q.shape, length_xy, dzf)
    gx, gy, gz = np.empty_like(q), np.empty_like(q), np.empty_like(q)
    L.oracle_gradient(_i(n), _d(Lxy), _d(dz), _d(q), _d(gx), _d(gy), _d(gz))
    return gx, gy, gz


def momentum_rhs(u, v, w, nu, length_xy, dzf):
    """A(u) + nu L(u) of Eq. up (conservative advection, no-slip walls)."""
    L = _bind_chan()
    u, v, w = _c(u), _c(v), _c(w)
    n, Lxy, dz = _chan_args(u.shape, length_xy, dzf)
    ru, rv, rw = np.empty_like(u), np.empty_like(u), np.empty_like(u)
    L.oracle_momentum_rhs(_i(n), _d(Lxy), _d(dz), float(nu), _d(u), _d(v), _d(w), _d(ru), _d(rv), _d(rw))
    return ru, rv, rw


def stable_dt(u, v, w, nu, cfl, length_xy, dzf):
    L = _bind_chan()
    u, v, w = _c(u), _c(v), _c(w)
    n, Lxy, dz = _chan_args(u.shape, length_xy, dzf)
    return float(L.oracle_stable_dt(_i(n), _d(Lxy), _d(dz), float(nu), float(cfl), _d(u), _d(v), _d(w)))


def project(u, v, w, length_xy, dzf, nthreads=0):
    """u - G L^-1 D u and the potential phi (pressure problem periodic x, y, Neumann z)."""
    L = _bind_chan()
    u, v, w = _c(u), _c(v), _c(w)
    n, Lxy, dz = _chan_args(u.shape, length_xy, dzf)
    uo, vo, wo, phi = (np.empty_like(u) for _ in range(4))
    rc = L.oracle_project(_i(n), _d(Lxy), _d(dz), _d(u), _d(v), _d(w), _d(uo), _d(vo), _d(wo), _d(phi), int(nthreads))
    if rc:
        raise ValueError(rc)
    return uo, vo, wo, phi


def rk3_step(u, v, w, p, nu, cfl, ubulk, length_xy, dzf, dt=0.0, nthreads=0):
    """One explicit low-storage RK3 fractional step; returns (u, v, w, p, dt) (copies)."""
    L = _bind_chan()
    u, v, w, p = (_c(a).copy() for a in (u, v, w, p))
    n, Lxy, dz = _chan_args(u.shape, length_xy, dzf)
    dt_out = ctypes.c_double()
    rc = L.oracle_rk3_step(_i(n), _d(Lxy), _d(dz), float(nu), float(cfl), float(ubulk), float(dt), _d(u), _d(v),
                           _d(w), _d(p), ctypes.byref(dt_out), int(nthreads))
    if rc:
        raise ValueError(rc)
    return u, v, w, p, float(dt_out.value)


def rk3_step_implicit(u, v, w, p, nu, cfl, ubulk, length_xy, dzf, dt=0.0, forcing=True, nthreads=0):
    """One RK3 step with Crank-Nicolson diffusion (Eq. up_id, Eq. up_id_2, the projection and the
    pressure update with -gamma nu dt/2 L Phi); returns (u, v, w, p, dt) (copies)."""
    L = _bind_chan()
    u, v, w, p = (_c(a).copy() for a in (u, v, w, p))
    n, Lxy, dz = _chan_args(u.shape, length_xy, dzf)
    dt_out = ctypes.c_double()
    rc = L.oracle_rk3_step_implicit(_i(n), _d(Lxy), _d(dz), float(nu), float(cfl), float(ubulk), int(bool(forcing)),
                                    float(dt), _d(u), _d(v), _d(w), _d(p), ctypes.byref(dt_out), int(nthreads))
    if rc:
        raise ValueError(rc)
    return u, v, w, p, float(dt_out.value)


# ---- the box: each direction periodic or bounded by no-slip walls, optional lid on the top z wall --
def _box_args(shape, walls, length_xy, dzf):
    n, Lxy, dz = _chan_args(shape, length_xy, dzf)
    return n, np.array([int(bool(x)) for x in walls], dtype=np.int32), Lxy, dz


def box_project(u, v, w, walls, length_xy, dzf, nthreads=0):
    L = _bind_chan()
    u, v, w = (_c(a).copy() for a in (u, v, w))
    n, wl, Lxy, dz = _box_args(u.shape, walls, length_xy, dzf)
    rc = L.oracle_box_project(_i(n), _i(wl), _d(Lxy), _d(dz), _d(u), _d(v), _d(w), int(nthreads))
    if rc:
        raise ValueError(rc)
    return u, v, w


def box_divergence(u, v, w, walls, length_xy, dzf):
    L = _bind_chan()
    u, v, w = _c(u), _c(v), _c(w)
    n, wl, Lxy, dz = _box_args(u.shape, walls, length_xy, dzf)
    out = np.empty_like(u)
    L.oracle_box_divergence(_i(n), _i(wl), _d(Lxy), _d(dz), _d(u), _d(v), _d(w), _d(out))
    return out


def box_operators(u, v, w, walls, length_xy, dzf, lid=0.0):
    """(advection, viscous operator) of the momentum equations, each a (u, v, w) triple."""
    L = _bind_chan()
    u, v, w = _c(u), _c(v), _c(w)
    n, wl, Lxy, dz = _box_args(u.shape, walls, length_xy, dzf)
    out = [np.empty_like(u) for _ in range(6)]
    L.oracle_box_operators(_i(n), _i(wl), float(lid), _d(Lxy), _d(dz), _d(u), _d(v), _d(w), *(_d(o) for o in out))
    return tuple(out[:3]), tuple(out[3:])


def box_rk3_step(u, v, w, p, walls, nu, length_xy, dzf, cfl=0.5, ubulk=0.0, forcing=False, dt=0.0, lid=0.0,
                 nthreads=0):
    """One explicit RK3 fractional step in the box; returns (u, v, w, p, dt) (copies)."""
    L = _bind_chan()
    u, v, w, p = (_c(a).copy() for a in (u, v, w, p))
    n, wl, Lxy, dz = _box_args(u.shape, walls, length_xy, dzf)
    dt_out = ctypes.c_double()
    rc = L.oracle_box_rk3_step(_i(n), _i(wl), float(lid), _d(Lxy), _d(dz), float(nu), float(cfl), float(ubulk),
                               int(bool(forcing)), float(dt), _d(u), _d(v), _d(w), _d(p), ctypes.byref(dt_out),
                               int(nthreads))
    if rc:
        raise ValueError(rc)
    return u, v, w, p, float(dt_out.value)
