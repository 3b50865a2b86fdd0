"""GPU parity of the Poisson path (through the C ABI) against the CPU oracle and library transforms."""
import itertools

import numpy as np
import pytest
import scipy.fft

import oracle
from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu

P, NN, DD = 0, 1, 2


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


def stream():
    import torch

    return int(torch.cuda.current_stream().cuda_stream)


def ref_forward(x, bc, axis):
    """Unnormalised forward transform in the library's slot order (scipy / numpy definitions)."""
    if bc == NN:
        return scipy.fft.dct(x, type=2, axis=axis)
    if bc == DD:
        return scipy.fft.dst(x, type=2, axis=axis)
    n = x.shape[axis]
    X = np.fft.rfft(x, axis=axis)
    X = np.moveaxis(X, axis, -1)
    out = np.empty(X.shape[:-1] + (n,))
    out[..., 0] = X[..., 0].real  # slot 0: X_0, slot 1: X_{n/2}, slots 2k, 2k+1: Re, Im X_k
    if n > 1:
        out[..., 1] = X[..., n // 2].real
    for k in range(1, n // 2):
        out[..., 2 * k] = X[..., k].real
        out[..., 2 * k + 1] = X[..., k].imag
    return np.moveaxis(out, -1, axis)


def slot_order(lam, bc):
    """Oracle eigenvalues (periodic basis columns k = 0, then cos/sin pairs 2k-1, 2k, then the
    Nyquist column last) rearranged into the library's slot order (slot 0 = mode 0, slot 1 = the
    Nyquist mode, slots 2k, 2k+1 = mode k).  Cosine / sine bases already match."""
    if bc != P or lam.shape[0] < 3:
        return lam
    n = lam.shape[0]
    out = np.empty_like(lam)
    out[0] = lam[0]
    out[1] = lam[n - 1]
    for k in range(1, n // 2):
        out[2 * k], out[2 * k + 1] = lam[2 * k - 1], lam[2 * k]
    return out


def make_plan(cans, n, bc, L=(1.0, 1.0), dzf=None, prec=0, sweeps=2, frac=0.01):
    o = cans.cans_opts_default()
    o.prec, o.max_sweeps, o.fp64_mode_fraction = prec, sweeps, frac
    _, h = cans.cans_poisson_plan(n, L, bc, dzf, o)
    return h


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------------------------------------
# transforms (x then y) against numpy / scipy
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bcx,bcy", list(itertools.product((P, NN, DD), (P, NN, DD))))
@pytest.mark.parametrize("n", [(16, 8, 3), (48, 96, 2), (1024, 64, 1), (2, 6, 2)])
def test_transform_xy_matches_library_transforms(cans, bcx, bcy, n):
    h = make_plan(cans, n, (bcx, bcy, NN))
    x = np.random.default_rng(1).standard_normal((n[2], n[1], n[0]))
    t = dev(x)
    assert cans.cans_transform_xy(h, t.data_ptr(), 1, stream()) == 0
    want = ref_forward(ref_forward(x, bcx, 2), bcy, 1)
    got = host(t)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    assert cans.cans_transform_xy(h, t.data_ptr(), -1, stream()) == 0
    back = host(t)
    assert np.abs(back - n[0] * n[1] * x).max() <= 1e-13 * n[0] * n[1] * np.abs(x).max()
    cans.cans_plan_destroy(h)


@pytest.mark.parametrize("bcx,bcy", list(itertools.product((P, NN, DD), (P, NN, DD))))
@pytest.mark.parametrize(
    "n", [(256, 512, 2), (1024, 128, 1), (512, 1024, 1), (64, 48, 2), (24, 256, 2), (32, 256, 3), (48, 1024, 2)]
)
def test_transform_xy_f32_matches_library_transforms(cans, bcx, bcy, n):
    """The mixed path's FP32 x/y passes: warp-per-line x kernels for N in {256, 512, 1024}, the
    lanes-across-x-slots y kernel for Ny in {256, 512, 1024} (Nx a multiple of 16; several tiles per
    plane and several planes), CTA-wide kernels otherwise; agreement to FP32 rounding."""
    import torch

    h = make_plan(cans, n, (bcx, bcy, NN), prec=1)
    x = np.random.default_rng(2).standard_normal((n[2], n[1], n[0]))
    t = dev(x)
    w = torch.empty(x.shape, dtype=torch.float32, device="cuda")
    assert cans.cans_transform_xy_f32(h, t.data_ptr(), w.data_ptr(), 1, stream()) == 0
    want = ref_forward(ref_forward(x, bcx, 2), bcy, 1)
    got = host(w).astype(np.float64)
    assert np.abs(got - want).max() <= 4e-6 * np.abs(want).max()
    assert cans.cans_transform_xy_f32(h, t.data_ptr(), w.data_ptr(), -1, stream()) == 0
    back = host(t)
    assert np.abs(back - n[0] * n[1] * x).max() <= 4e-6 * n[0] * n[1] * np.abs(x).max()
    cans.cans_plan_destroy(h)


@pytest.mark.parametrize("n", [(512, 256, 2), (48, 32, 3)])
def test_transform_xy_f32_special_inputs(cans, n):
    """Inputs the integer double -> float rounding leaves to the hardware conversion (exact zeros,
    values below the float range, signed zeros) mixed into ordinary ones: the forward x-y transform
    of the float-rounded field, to FP32 rounding."""
    import torch

    h = make_plan(cans, n, (P, NN, NN), prec=1)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((n[2], n[1], n[0]))
    sel = rng.random(x.shape)
    x[sel < 0.02] = 0.0
    x[(sel >= 0.02) & (sel < 0.03)] = 1e-300
    x[(sel >= 0.03) & (sel < 0.035)] = -0.0
    x[(sel >= 0.035) & (sel < 0.04)] = 3e-39  # a float subnormal
    t = dev(x)
    w = torch.empty(x.shape, dtype=torch.float32, device="cuda")
    assert cans.cans_transform_xy_f32(h, t.data_ptr(), w.data_ptr(), 1, stream()) == 0
    xf = x.astype(np.float32).astype(np.float64)
    want = ref_forward(ref_forward(xf, P, 2), NN, 1)
    got = host(w).astype(np.float64)
    assert np.abs(got - want).max() <= 4e-6 * np.abs(want).max()
    cans.cans_plan_destroy(h)


def test_transform_xy_f32_rejects_fp64_plans(cans):
    import torch

    h = make_plan(cans, (32, 32, 2), (P, P, NN), prec=0)
    t = torch.zeros((2, 32, 32), dtype=torch.float64, device="cuda")
    w = torch.zeros((2, 32, 32), dtype=torch.float32, device="cuda")
    assert cans.cans_transform_xy_f32(h, t.data_ptr(), w.data_ptr(), 1, stream()) != 0
    cans.cans_plan_destroy(h)


@pytest.mark.parametrize("bc", [(P, P, NN), (NN, DD, NN), (DD, P, DD)])
def test_mixed_refined_warp_engine_sizes(cans, bc):
    """Refined mixed solve on a shape every fused pass of which runs on the warp-per-line kernels."""
    n = (256, 128, 12)
    dzf = I.tanh_dzf(12, 1.6)
    case = I.case_modes(n=n)
    case.bc = bc
    case.dzf = dzf
    f = I.rhs_host(case)
    p, st, info = solve_gpu(cans, f, n, bc, (1.0, 1.0), dzf, prec=1, sweeps=2, info=True)
    ref = oracle.poisson_solve(f, bc, (1.0, 1.0), dzf)
    res = oracle.relative_residual(p, f, bc, (1.0, 1.0), dzf)
    floor = oracle.relative_residual(ref, f, bc, (1.0, 1.0), dzf)
    assert res <= max(1e-12, 2 * floor), (res, floor, info)
    assert rel(p, ref) <= 1e-11
    assert st == 0


# ---------------------------------------------------------------------------------------------
# z tridiagonal pass against the oracle's rows and Thomas
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("nz", [1, 2, 5, 33, 64, 200, 512])
@pytest.mark.parametrize("bcz", [NN, DD])
def test_zsolve_matches_thomas(cans, nz, bcz):
    n = (48, 6, nz)
    bc = (P, DD, bcz)
    dzf = I.tanh_dzf(nz, 1.6) if nz > 1 else np.ones(1)
    h = make_plan(cans, n, bc, (1.3, 0.9), dzf)
    g = np.random.default_rng(nz).standard_normal((nz, n[1], n[0]))
    t = dev(g)
    assert cans.cans_zsolve(h, t.data_ptr(), stream()) == 0
    got = host(t)
    lx = slot_order(oracle.eigenbasis(bc[0], n[0])[1], bc[0])
    ly = slot_order(oracle.eigenbasis(bc[1], n[1])[1], bc[1])
    mux = lx / (1.3 / n[0]) ** 2
    muy = ly / (0.9 / n[1]) ** 2
    a, b, c = oracle.z_rows(bcz, dzf)
    want = np.empty_like(g)
    for j in range(n[1]):
        for i in range(n[0]):
            want[:, j, i] = oracle.thomas(a, b + mux[i] + muy[j], c, g[:, j, i])
    assert rel(got, want) < 1e-12
    cans.cans_plan_destroy(h)


def test_plan_eigenvalues_match_oracle(cans):
    n = (24, 12, 4)
    h = make_plan(cans, n, (P, DD, NN), (2.0, 3.0))
    mx, my = cans.cans_plan_eigenvalues(h, 24, 12)
    lx = slot_order(oracle.eigenbasis(P, 24)[1], P)
    ly = slot_order(oracle.eigenbasis(DD, 12)[1], DD)
    assert np.abs(mx - lx / (2.0 / 24) ** 2).max() < 1e-12 * np.abs(mx).max()
    assert np.abs(my - ly / (3.0 / 12) ** 2).max() < 1e-12 * np.abs(my).max()
    cans.cans_plan_destroy(h)


# ---------------------------------------------------------------------------------------------
# full FP64 solve against the oracle
# ---------------------------------------------------------------------------------------------
def solve_gpu(cans, f, n, bc, L, dzf, prec=0, sweeps=2, frac=0.01, info=False):
    import torch

    h = make_plan(cans, n, bc, L, dzf, prec, sweeps, frac)
    nbytes = cans.cans_poisson_workspace_size(h)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    wp = (ws.data_ptr() + 255) // 256 * 256 if nbytes else 0
    ft = dev(f)
    pt = torch.full_like(ft, float("nan"))
    buf = np.zeros(sweeps + 2) if info else None
    st = cans.cans_poisson_solve(h, ft.data_ptr(), pt.data_ptr(), wp, stream(), buf)
    p = host(pt)
    cans.cans_plan_destroy(h)
    return p, st, buf


def test_uniform32_fp64_matches_oracle(cans):
    case = I.case_uniform32()
    f = I.rhs_host(case)
    p, st, info = solve_gpu(cans, f, case.n, case.bc, case.length_xy, case.dzf, info=True)
    assert st == 0
    ref = oracle.poisson_solve(f, case.bc, case.length_xy, case.dzf)
    assert rel(p, ref) <= 1e-12
    assert oracle.relative_residual(p, f, case.bc, case.length_xy, case.dzf) <= 1e-13
    assert info[0] <= 1e-13  # the library's own residual report agrees


def test_dense_lu_8cubed_copy(cans):
    from tests.test_oracle_pins import dense_operator, dense_solve, volumes

    case = I.case_uniform32(n=(8, 8, 8))
    f = I.rhs_host(case)
    A = dense_operator(case.n, case.bc, case.length_xy, case.dzf)
    ref = dense_solve(A, f.ravel(), volumes(case.n, case.length_xy, case.dzf)).reshape(f.shape)
    p, st, _ = solve_gpu(cans, f, case.n, case.bc, case.length_xy, case.dzf)
    assert st == 0 and rel(p, ref) <= 1e-12


BC_CASES = [(bx, by, bz) for bx in (P, NN, DD) for by in (P, NN, DD) for bz in (P, NN, DD)]


@pytest.mark.parametrize("bc", BC_CASES)
def test_fp64_solve_all_boundary_conditions(cans, bc):
    nz = 20 if bc[2] != P else 24  # a ragged z segment; a periodic z needs N/2 = 2^a 3^b
    n = (48, 24, nz)  # radix-3 lengths, x tiles with a tail
    dzf = I.tanh_dzf(nz, 1.8) if bc[2] != P else I.uniform_dzf(nz)
    L = (1.5, 0.75)
    f = np.random.default_rng(sum(bc)).uniform(-1, 1, (nz, 24, 48))
    if DD not in bc:
        f = I.weighted_mean_removed(f, dzf)
    p, st, _ = solve_gpu(cans, f, n, bc, L, dzf)
    assert st == 0
    ref = oracle.poisson_solve(f, bc, L, dzf)
    assert rel(p, ref) <= 1e-12


@pytest.mark.parametrize(
    "n,bc",
    [
        ((1, 1, 17), (P, P, DD)),  # pure z problem
        ((1, 8, 8), (NN, P, NN)),  # one x cell
        ((8, 1, 8), (DD, NN, NN)),  # one y cell
        ((8, 8, 1), (P, DD, NN)),  # one z cell
        ((2, 2, 2), (P, P, NN)),  # smallest even lengths, singular
        ((64, 96, 31), (P, NN, DD)),  # radix 3 in y, odd Nz
        ((16, 16, 512), (P, P, NN)),  # 16 rows per lane
        ((8, 6, 1), (P, P, P)),  # one periodic z cell
        ((16, 12, 96), (DD, P, P)),  # periodic z, radix 3
    ],
)
def test_fp64_solve_edge_shapes(cans, n, bc):
    nx, ny, nz = n
    dzf = I.tanh_dzf(nz, 1.4) if (nz > 2 and bc[2] != P) else I.uniform_dzf(nz)
    f = np.random.default_rng(nx + 7 * ny + 13 * nz).uniform(-1, 1, (nz, ny, nx))
    if DD not in bc:
        f = I.weighted_mean_removed(f, dzf)
    p, st, _ = solve_gpu(cans, f, n, bc, (1.0, 1.0), dzf)
    assert st == 0
    ref = oracle.poisson_solve(f, bc, (1.0, 1.0), dzf)
    assert rel(p, ref) <= 1e-12


def test_in_place_fp64(cans):
    import torch

    case = I.case_channel(n=(64, 32, 16))
    f = I.rhs_host(case)
    h = make_plan(cans, case.n, case.bc, case.length_xy, case.dzf)
    t = dev(f)
    assert cans.cans_poisson_solve(h, t.data_ptr(), t.data_ptr(), 0, stream(), None) == 0
    ref = oracle.poisson_solve(f, case.bc, case.length_xy, case.dzf)
    assert rel(host(t), ref) <= 1e-12
    cans.cans_plan_destroy(h)


def test_incompatible_rhs_is_reported(cans):
    case = I.case_uniform32(n=(16, 16, 8))
    f = I.rhs_host(case) + 0.3  # non-zero mean on a singular problem
    p, st, info = solve_gpu(cans, f, case.n, case.bc, case.length_xy, case.dzf, info=True)
    assert st == -5
    # the returned p still solves the compatible part and has zero weighted mean
    fc = I.weighted_mean_removed(f, case.dzf)
    assert rel(p, oracle.poisson_solve(fc, case.bc, case.length_xy, case.dzf)) <= 1e-12


# ---------------------------------------------------------------------------------------------
# mixed precision + refinement
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc", [(P, P, NN), (P, DD, NN), (NN, DD, DD), (DD, NN, NN), (P, P, P), (NN, DD, P)])
def test_mixed_refined_reaches_fp64_accuracy(cans, bc):
    n = (64, 48, 40) if bc[2] != P else (64, 48, 48)
    dzf = I.tanh_dzf(40, 1.8) if bc[2] != P else I.uniform_dzf(48)
    case = I.case_modes(n=n)
    case.bc = bc
    case.dzf = dzf
    f = I.rhs_host(case)
    p, st, info = solve_gpu(cans, f, n, bc, (1.0, 1.0), dzf, prec=1, sweeps=2, info=True)
    ref = oracle.poisson_solve(f, bc, (1.0, 1.0), dzf)
    res = oracle.relative_residual(p, f, bc, (1.0, 1.0), dzf)
    floor = oracle.relative_residual(ref, f, bc, (1.0, 1.0), dzf)
    d = p - ref
    w = dzf[:, None, None] * np.ones_like(d)
    offset = float((d * w).sum() / w.sum())
    diag = dict(res=res, floor=floor, info=info, rel=rel(p, ref), offset_rel=offset / np.abs(ref).max(),
                rel_without_offset=rel(p - offset, ref))
    assert res <= max(1e-12, 2 * floor), diag
    assert rel(p, ref) <= 1e-11, diag
    assert info[0] > info[1], info
    assert st == 0


def test_mixed_refined_with_special_rhs_values(cans):
    """A right-hand side with exact zeros, signed zeros and values below the float range (the inputs
    the residual stencil's integer split of f leaves to its general path): the mixed solve still
    reaches the FP64 accuracy of the oracle."""
    bc = (P, DD, NN)
    n = (64, 48, 40)
    dzf = I.tanh_dzf(40, 1.8)
    case = I.case_modes(n=n)
    case.bc = bc
    case.dzf = dzf
    f = I.rhs_host(case).copy()
    sel = np.random.default_rng(6).random(f.shape)
    f[sel < 0.03] = 0.0
    f[(sel >= 0.03) & (sel < 0.04)] = -0.0
    f[(sel >= 0.04) & (sel < 0.05)] = 1e-300
    p, st, info = solve_gpu(cans, f, n, bc, (1.0, 1.0), dzf, prec=1, sweeps=2, info=True)
    ref = oracle.poisson_solve(f, bc, (1.0, 1.0), dzf)
    res = oracle.relative_residual(p, f, bc, (1.0, 1.0), dzf)
    floor = oracle.relative_residual(ref, f, bc, (1.0, 1.0), dzf)
    assert res <= max(1e-12, 2 * floor), (res, floor, info)
    assert rel(p, ref) <= 1e-11
    assert st == 0


def test_mixed_first_solve_only(cans):
    case = I.case_modes(n=(32, 32, 16))
    f = I.rhs_host(case)
    p, st, info = solve_gpu(cans, f, case.n, case.bc, case.length_xy, case.dzf, prec=1, sweeps=0, info=True)
    ref = oracle.poisson_solve(f, case.bc, case.length_xy, case.dzf)
    assert rel(p, ref) < 1e-4  # FP32 transforms alone
    assert st == -6  # tolerance 1e-12 not reached without refinement


def test_autotuned_plan_matches_oracle(cans, tmp_path, monkeypatch):
    """opts.autotune = 1 picks tile shapes by timing; results stay exact and the cache file is written."""
    import torch

    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("CANS_AUTOTUNE_CACHE", str(cache))
    case = I.case_channel(n=(128, 64, 48))
    f = I.rhs_host(case)
    ref = oracle.poisson_solve(f, case.bc, case.length_xy, case.dzf)
    for prec in (0, 1):
        o = cans.cans_opts_default()
        o.prec, o.max_sweeps, o.autotune = prec, 2, 1
        _, h = cans.cans_poisson_plan(case.n, case.length_xy, case.bc, case.dzf, o)
        nbytes = cans.cans_poisson_workspace_size(h)
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        wp = (ws.data_ptr() + 255) // 256 * 256 if nbytes else 0
        ft = dev(f)
        pt = torch.empty_like(ft)
        assert cans.cans_poisson_solve(h, ft.data_ptr(), pt.data_ptr(), wp, stream(), None) == 0
        assert rel(host(pt), ref) <= (1e-12 if prec == 0 else 1e-11)
        cans.cans_plan_destroy(h)
    lines = cache.read_text().strip().splitlines()
    # key, then lines per CTA of x and y, of the spectral z pass, the z tile width, the TMA z kernel flag
    assert len(lines) == 2 and all(len(l.split()) == 6 for l in lines)
