// Test infrastructure -- NOT part of the product path.
//
// A plain, slow, obviously correct CPU implementation of what the pressure-Poisson hot path computes:
// the exact solution of the second-order, 7-point, staggered finite-difference Poisson equation
// (eq. poi, "FFT-based Poisson solver" subsection of Numerical method) reached the way the paper
// describes it (eq. poi_reduced): diagonalise the x and y operators with their eigenvectors, then
// solve one tridiagonal system along z per (x, y) mode by Gauss elimination.
//
// The eigenvectors are written out as dense orthonormal bases (closed-form cos/sin columns), and the
// transforms are dense matrix products -- no FFT, no Makhoul tricks, no blocking.  Every routine is a
// template over the scalar type so the same source runs in double, long double and __float128.
//
// Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load this library.
// It shares no code with the CUDA path.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <quadmath.h>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

enum { BC_P = 0, BC_NN = 1, BC_DD = 2, BC_ND = 3, BC_DN = 4 };
// ND / DN: Neumann at the low wall and Dirichlet at the high wall, or the reverse -- the remaining
// cell-centred wall combinations of the Numerical method's transform list.  The wall rule of each
// end of a direction:
inline int bc_low(int bc) { return (bc == BC_ND) ? BC_NN : (bc == BC_DN ? BC_DD : bc); }
inline int bc_high(int bc) { return (bc == BC_ND) ? BC_DD : (bc == BC_DN ? BC_NN : bc); }
inline bool has_dirichlet(int bc) { return bc == BC_DD || bc == BC_ND || bc == BC_DN; }

// Deliberate-mistake switch used only by the mutation tests (tests/test_oracle_mutations.py): each
// value plants one plausible error so the tests can show that some pin catches it.  0 = correct.
int g_fault = 0;

typedef __float128 quad;

// ---- scalar helpers for the three precisions --------------------------------------------------
inline double sin_(double x) { return std::sin(x); }
inline long double sin_(long double x) { return sinl(x); }
inline quad sin_(quad x) { return sinq(x); }
inline double cos_(double x) { return std::cos(x); }
inline long double cos_(long double x) { return cosl(x); }
inline quad cos_(quad x) { return cosq(x); }
inline double sqrt_(double x) { return std::sqrt(x); }
inline long double sqrt_(long double x) { return sqrtl(x); }
inline quad sqrt_(quad x) { return sqrtq(x); }
template <typename T> T pi_();
template <> double pi_<double>() { return 3.14159265358979323846264338327950288; }
template <> long double pi_<long double>() { return 3.14159265358979323846264338327950288L; }
template <> quad pi_<quad>() { return acosq((quad)-1); }

// ---- grid (Validation section: x, y uniform; z cell widths dzf may be non-uniform) ---------------
// z centres sit half-way between faces; dzc[k+1] is the centre-to-centre distance between cells k
// and k+1 (stored with an offset of one so that dzc[0] is the wall ghost distance below cell 0 and
// dzc[nz] the one above cell nz-1).  At a wall the ghost cell mirrors the first interior cell, so
// the ghost distance equals the wall cell's width.  A periodic z wraps.
//
// Face grid (faces = true; the staggered w of the marker-and-cell grid, Numerical method, solved
// implicitly by Eq. up_id_2): the unknowns sit on the nz = ncells - 1 interior faces, unknown k on
// the face between cells k and k+1; w = 0 on both wall faces.  Its second difference at face k is
//   [ (w_{k+1} - w_k) / dzf_{k+1} - (w_k - w_{k-1}) / dzf_k ] / mid_k,
// mid_k = (dzf_k + dzf_{k+1}) / 2 the distance between the centres of the two cells, w_{-1} = w_nz = 0.
template <typename T>
struct ZGrid {
  int nz, bc;
  bool faces;
  std::vector<T> dzf, dzc;  // cell grid: dzf[k], k=0..nz-1; dzc[k], k=0..nz (see above)
  std::vector<T> cell, mid;  // face grid: the ncells cell widths and the nz centre distances mid_k
  ZGrid(int ncells, int bc_, const double* dzf_in, bool faces_ = false)
      : nz(ncells - (faces_ ? 1 : 0)), bc(bc_), faces(faces_), dzf(nz), dzc(nz + 1) {
    if (faces) {
      cell.resize(ncells);
      mid.resize(nz);
      for (int k = 0; k < ncells; ++k) cell[k] = (T)dzf_in[k];
      for (int k = 0; k < nz; ++k) mid[k] = (cell[k] + cell[k + 1]) / 2;
      for (int k = 0; k < nz; ++k) dzf[k] = mid[k];  // control-volume widths (weights of the mean)
      return;
    }
    for (int k = 0; k < nz; ++k) dzf[k] = (T)dzf_in[k];
    for (int k = 1; k < nz; ++k) dzc[k] = (dzf[k - 1] + dzf[k]) / 2;
    if (bc == BC_P) {
      dzc[0] = dzc[nz] = (dzf[nz - 1] + dzf[0]) / 2;
    } else {
      dzc[0] = dzf[0];
      dzc[nz] = dzf[nz - 1];
    }
  }
};

// ---- the operator L_h of eq. poi, with the ghost rules of each boundary condition -----------------
// One direction, uniform spacing h: (q[i-1] - 2 q[i] + q[i+1]) / h^2 with ghosts:
// periodic wraps; Neumann-Neumann q[-1] = q[0]; Dirichlet-Dirichlet q[-1] = -q[0] (wall half-way
// between ghost and first cell), likewise at the far end.
template <typename T>
inline T ghost(int bc, T inner, T wrap) {
  if (bc == BC_P) return wrap;
  if (bc == BC_NN) return inner;
  return -inner;
}

// (L_h + shift) p: the Helmholtz form of Eq. up_id_2 when shift != 0.
template <typename T>
void apply_laplacian(const int n[3], const T len_xy[2], const int bc[3], const ZGrid<T>& zg, const T* p, T* out,
                     int nthreads, T shift = 0) {
  const int nx = n[0], ny = n[1], nz = n[2];
  const T dx = len_xy[0] / nx, dy = len_xy[1] / ny;
  const T idx2 = 1 / (dx * dx), idy2 = 1 / (dy * dy);
  const size_t sx = 1, sy = nx, sz = (size_t)nx * ny;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int k = 0; k < nz; ++k) {
    for (int j = 0; j < ny; ++j) {
      for (int i = 0; i < nx; ++i) {
        const size_t c = i * sx + j * sy + k * sz;
        const T pc = p[c];
        const T xm = (i > 0) ? p[c - sx] : ghost<T>(bc_low(bc[0]), pc, p[c + (nx - 1) * sx]);
        const T xp = (i < nx - 1) ? p[c + sx] : ghost<T>(bc_high(bc[0]), pc, p[c - (nx - 1) * sx]);
        const T ym = (j > 0) ? p[c - sy] : ghost<T>(bc_low(bc[1]), pc, p[c + (ny - 1) * sy]);
        const T yp = (j < ny - 1) ? p[c + sy] : ghost<T>(bc_high(bc[1]), pc, p[c - (ny - 1) * sy]);
        const T zm = (k > 0) ? p[c - sz] : ghost<T>(bc_low(bc[2]), pc, p[c + (nz - 1) * sz]);
        const T zp = (k < nz - 1) ? p[c + sz] : ghost<T>(bc_high(bc[2]), pc, p[c - (nz - 1) * sz]);
        const T lx = (xm - 2 * pc + xp) * idx2;
        const T ly = (ym - 2 * pc + yp) * idy2;
        T lz;
        if (zg.faces) {  // w on faces, zero on the wall faces
          const T wm = (k > 0) ? p[c - sz] : T(0), wp = (k < nz - 1) ? p[c + sz] : T(0);
          lz = ((wp - pc) / zg.cell[k + 1] - (pc - wm) / zg.cell[k]) / zg.mid[k];
        } else {
          // z: (1/dzf_k) [ (p_{k+1}-p_k)/dzc_{k+1/2} - (p_k-p_{k-1})/dzc_{k-1/2} ]  (non-uniform z)
          T up = (zp - pc) / zg.dzc[k + 1];
          T dn = (pc - zm) / zg.dzc[k];
          if (g_fault == 1) dn = (pc - zm) / zg.dzc[k + 1];  // planted: wrong metric index
          lz = (up - dn) / zg.dzf[k];
        }
        out[c] = lx + ly + lz + shift * pc;
      }
    }
  }
}

// ---- orthonormal eigenbases of the 1-D operators (the discrete operator F of eq. poi_reduced) -----
// Column m of E is an eigenvector of the 1-D second-difference operator of that boundary condition
// (unit spacing) with eigenvalue lam[m]; E is stored row-major, E[i*n + m].
//   periodic : 1/sqrt(n); sqrt(2/n) cos(2 pi k i/n), sqrt(2/n) sin(2 pi k i/n) for 1 <= k < n/2
//              (columns 2k-1 and 2k); (-1)^i/sqrt(n) if n is even (last column).
//              lam = -4 sin^2(pi k/n), which equals 2(cos(2 pi k/n) - 1).
//   Neumann  : sqrt(2/n) c_m cos(pi m (i+1/2)/n), c_0 = 1/sqrt(2); lam = -4 sin^2(pi m/(2n)).
//   Dirichlet: sqrt(2/n) c_m sin(pi (m+1)(i+1/2)/n), c_{n-1} = 1/sqrt(2); lam = -4 sin^2(pi (m+1)/(2n)).
//   Neumann-Dirichlet: sqrt(2/n) cos(pi (m+1/2)(i+1/2)/n); Dirichlet-Neumann: sqrt(2/n) sin(pi (m+1/2)(i+1/2)/n);
//              both lam = -4 sin^2(pi (2m+1)/(4n)) (quarter waves: zero slope at one wall, zero value
//              half a cell beyond the other).
template <typename T>
void eigenbasis(int bc, int n, std::vector<T>& E, std::vector<T>& lam) {
  E.assign((size_t)n * n, T(0));
  lam.assign(n, T(0));
  const T pi = pi_<T>();
  const T s2n = sqrt_(T(2) / n), s1n = sqrt_(T(1) / n);
  if (bc == BC_P) {
    for (int i = 0; i < n; ++i) E[(size_t)i * n + 0] = s1n;
    lam[0] = 0;
    const int kmax = (n % 2 == 0) ? n / 2 - 1 : (n - 1) / 2;
    for (int k = 1; k <= kmax; ++k) {
      for (int i = 0; i < n; ++i) {
        const T th = 2 * pi * T(k) * T(i) / T(n);
        E[(size_t)i * n + 2 * k - 1] = s2n * cos_(th);
        E[(size_t)i * n + 2 * k] = s2n * sin_(th);
      }
      const T s = sin_(pi * T(k) / T(n));
      lam[2 * k - 1] = lam[2 * k] = -4 * s * s;
    }
    if (n % 2 == 0) {
      for (int i = 0; i < n; ++i) E[(size_t)i * n + n - 1] = (i % 2 == 0) ? s1n : -s1n;
      lam[n - 1] = -4;
    }
  } else if (bc == BC_NN) {
    for (int m = 0; m < n; ++m) {
      const T cm = (m == 0) ? sqrt_(T(0.5)) : T(1);
      for (int i = 0; i < n; ++i) E[(size_t)i * n + m] = s2n * cm * cos_(pi * T(m) * (T(i) + T(0.5)) / T(n));
      const T s = sin_(pi * T(m) / (2 * T(n)));
      lam[m] = -4 * s * s;
    }
  } else if (bc == BC_DD) {
    for (int m = 0; m < n; ++m) {
      const T cm = (m == n - 1) ? sqrt_(T(0.5)) : T(1);
      for (int i = 0; i < n; ++i) E[(size_t)i * n + m] = s2n * cm * sin_(pi * T(m + 1) * (T(i) + T(0.5)) / T(n));
      const T s = sin_(pi * T(m + 1) / (2 * T(n)));
      lam[m] = -4 * s * s;
    }
  } else {  // BC_ND, BC_DN
    for (int m = 0; m < n; ++m) {
      for (int i = 0; i < n; ++i) {
        const T th = pi * (T(m) + T(0.5)) * (T(i) + T(0.5)) / T(n);
        E[(size_t)i * n + m] = s2n * ((bc == BC_ND) ? cos_(th) : sin_(th));
      }
      const T s = sin_(pi * T(2 * m + 1) / (4 * T(n)));
      lam[m] = -4 * s * s;
    }
  }
  if (g_fault == 2) {  // planted: eigenvalue of the neighbouring mode
    std::vector<T> l2(lam);
    for (int m = 0; m + 1 < n; ++m) lam[m] = l2[m + 1];
  }
}

// ---- z tridiagonal rows of L_h for one (x, y) mode: a_k p_{k-1} + b_k p_k + c_k p_{k+1} ------------
template <typename T>
void z_rows(const ZGrid<T>& zg, std::vector<T>& a, std::vector<T>& b, std::vector<T>& c) {
  const int nz = zg.nz;
  a.assign(nz, T(0));
  b.assign(nz, T(0));
  c.assign(nz, T(0));
  if (zg.faces) {  // the face operator above, the zero wall values dropped from the rows
    for (int k = 0; k < nz; ++k) {
      a[k] = (k > 0) ? 1 / (zg.cell[k] * zg.mid[k]) : T(0);
      c[k] = (k < nz - 1) ? 1 / (zg.cell[k + 1] * zg.mid[k]) : T(0);
      b[k] = -(1 / (zg.cell[k] * zg.mid[k]) + 1 / (zg.cell[k + 1] * zg.mid[k]));
    }
    return;
  }
  for (int k = 0; k < nz; ++k) {
    a[k] = 1 / (zg.dzf[k] * zg.dzc[k]);
    c[k] = 1 / (zg.dzf[k] * zg.dzc[k + 1]);
    b[k] = -(a[k] + c[k]);
  }
  if (zg.bc != BC_P) {
    // Neumann end: the ghost equals the wall cell and that flux vanishes; Dirichlet end: the ghost is
    // minus the wall cell
    b[0] += (bc_low(zg.bc) == BC_NN) ? a[0] : -a[0];
    b[nz - 1] += (bc_high(zg.bc) == BC_NN) ? c[nz - 1] : -c[nz - 1];
  }
  if (zg.bc != BC_P) {
    a[0] = 0;
    c[nz - 1] = 0;
  }
}

// Plain Gauss elimination without pivoting (Thomas) for a_k x_{k-1} + b_k x_k + c_k x_{k+1} = d_k.
template <typename T>
void thomas(int n, const T* a, const T* b, const T* c, const T* d, T* x) {
  std::vector<T> cp(n), dp(n);
  cp[0] = c[0] / b[0];
  dp[0] = d[0] / b[0];
  for (int k = 1; k < n; ++k) {
    const T m = b[k] - a[k] * cp[k - 1];
    cp[k] = c[k] / m;
    dp[k] = (d[k] - a[k] * dp[k - 1]) / m;
  }
  x[n - 1] = dp[n - 1];
  for (int k = n - 2; k >= 0; --k) x[k] = dp[k] - cp[k] * x[k + 1];
}

// ---- the direct solver (eq. poi_reduced) ---------------------------------------------------------
// fhat = (Ex^T (x) Ey^T) f;  for every (mx, my): (A_z + mu I) phat = fhat with
// mu = lam_x/dx^2 + lam_y/dy^2;  p = (Ex (x) Ey) phat.
// If z is periodic (uniform only) the z direction is diagonalised too.
// Singular case (x, y, z all periodic or Neumann): the (0,0) z-system is singular; its last equation
// is dropped with phat_{nz-1} = 0, and the result is shifted to zero dzf-weighted mean, which makes
// the cell-volume-weighted mean of p zero.
// With a Helmholtz shift (Eq. up_id_2) every diagonal gets + shift and no mode is singular.
template <typename T>
int poisson_solve(const int n[3], const T len_xy[2], const int bc[3], const ZGrid<T>& zg, const T* f, T* p,
                  int nthreads, T shift = 0) {
  const int nx = n[0], ny = n[1], nz = n[2];
  const size_t plane = (size_t)nx * ny;
  std::vector<T> Ex, lx, Ey, ly, Ez, lz;
  eigenbasis<T>(bc[0], nx, Ex, lx);
  eigenbasis<T>(bc[1], ny, Ey, ly);
  const T dx = len_xy[0] / nx, dy = len_xy[1] / ny;
  std::vector<T> hat(plane * nz);

  // forward: per z-plane, hat = Ey^T F Ex with F the [ny][nx] plane
#pragma omp parallel num_threads(nthreads)
  {
    std::vector<T> tmp(plane);
#pragma omp for schedule(static)
    for (int k = 0; k < nz; ++k) {
      const T* F = f + k * plane;
      std::fill(tmp.begin(), tmp.end(), T(0));
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          const T s = F[(size_t)j * nx + i];
          const T* e = &Ex[(size_t)i * nx];
          T* t = &tmp[(size_t)j * nx];
          for (int m = 0; m < nx; ++m) t[m] += s * e[m];
        }
      T* H = hat.data() + k * plane;
      std::fill(H, H + plane, T(0));
      for (int my = 0; my < ny; ++my)
        for (int j = 0; j < ny; ++j) {
          const T s = Ey[(size_t)j * ny + my];
          const T* t = &tmp[(size_t)j * nx];
          T* h = &H[(size_t)my * nx];
          for (int m = 0; m < nx; ++m) h[m] += s * t[m];
        }
    }
  }

  const bool singular = !has_dirichlet(bc[0]) && !has_dirichlet(bc[1]) && !has_dirichlet(bc[2]) && shift == 0;
  if (bc[2] == BC_P) {
    // uniform periodic z: diagonalise z as well (checked by the caller)
    eigenbasis<T>(BC_P, nz, Ez, lz);
    const T dz = zg.dzf[0];
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long long col = 0; col < (long long)plane; ++col) {
      const int mx = (int)(col % nx), my = (int)(col / nx);
      const T mu = lx[mx] / (dx * dx) + ly[my] / (dy * dy);
      std::vector<T> g(nz), q(nz, T(0));
      for (int k = 0; k < nz; ++k) g[k] = hat[col + k * plane];
      for (int mz = 0; mz < nz; ++mz) {
        T s = 0;
        for (int k = 0; k < nz; ++k) s += Ez[(size_t)k * nz + mz] * g[k];
        const T den = mu + lz[mz] / (dz * dz) + shift;
        q[mz] = (singular && mx == 0 && my == 0 && mz == 0) ? T(0) : s / den;
      }
      for (int k = 0; k < nz; ++k) {
        T s = 0;
        for (int mz = 0; mz < nz; ++mz) s += Ez[(size_t)k * nz + mz] * q[mz];
        hat[col + k * plane] = s;
      }
    }
  } else {
    std::vector<T> a, b, c;
    z_rows<T>(zg, a, b, c);
    T wsum = 0;
    for (int k = 0; k < nz; ++k) wsum += zg.dzf[k];
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (long long col = 0; col < (long long)plane; ++col) {
      const int mx = (int)(col % nx), my = (int)(col / nx);
      const T mu = lx[mx] / (dx * dx) + ly[my] / (dy * dy);
      std::vector<T> bb(nz), d(nz), x(nz);
      for (int k = 0; k < nz; ++k) {
        bb[k] = b[k] + mu + shift;
        d[k] = hat[col + k * plane];
      }
      if (singular && mx == 0 && my == 0) {
        x[nz - 1] = 0;
        if (nz > 1) thomas<T>(nz - 1, a.data(), bb.data(), c.data(), d.data(), x.data());
        T m = 0;
        for (int k = 0; k < nz; ++k) m += zg.dzf[k] * x[k];
        m /= wsum;
        for (int k = 0; k < nz; ++k) x[k] -= m;
      } else {
        thomas<T>(nz, a.data(), bb.data(), c.data(), d.data(), x.data());
      }
      for (int k = 0; k < nz; ++k) hat[col + k * plane] = x[k];
    }
  }

  // inverse: per z-plane, P = Ey H Ex^T
#pragma omp parallel num_threads(nthreads)
  {
    std::vector<T> tmp(plane);
#pragma omp for schedule(static)
    for (int k = 0; k < nz; ++k) {
      const T* H = hat.data() + k * plane;
      std::fill(tmp.begin(), tmp.end(), T(0));
      for (int j = 0; j < ny; ++j)
        for (int my = 0; my < ny; ++my) {
          const T s = Ey[(size_t)j * ny + my];
          const T* h = &H[(size_t)my * nx];
          T* t = &tmp[(size_t)j * nx];
          for (int m = 0; m < nx; ++m) t[m] += s * h[m];
        }
      T* P = p + k * plane;
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          const T* e = &Ex[(size_t)i * nx];
          const T* t = &tmp[(size_t)j * nx];
          T s = 0;
          if (g_fault == 3) {  // planted: transposed basis on the way back
            for (int m = 0; m < nx; ++m) s += Ex[(size_t)m * nx + i] * t[m];
          } else {
            for (int m = 0; m < nx; ++m) s += e[m] * t[m];
          }
          P[(size_t)j * nx + i] = s;
        }
    }
  }
  return 0;
}

int check_args(const int n[3], const int bc[3], const double* dzf) {
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 1) return -1;
    if (bc[d] < 0 || bc[d] > 4) return -1;
  }
  for (int k = 0; k < n[2]; ++k)
    if (!(dzf[k] > 0) || !std::isfinite(dzf[k])) return -1;
  if (bc[2] == BC_P)
    for (int k = 1; k < n[2]; ++k)
      if (dzf[k] != dzf[0]) return -2;  // periodic z must be uniform
  return 0;
}

// n[2] counts the cells of dzf; the unknowns along z are n[2] (cell grid) or n[2] - 1 (face grid).
template <typename T>
int solve_t(const int n[3], const double len_xy[2], const int bc[3], const double* dzf, const double* f, double* p,
            int nthreads, double shift = 0, int faces = 0) {
  ZGrid<T> zg(n[2], bc[2], dzf, faces != 0);
  const int nu[3] = {n[0], n[1], zg.nz};
  const size_t N = (size_t)n[0] * n[1] * zg.nz;
  std::vector<T> ft(N), pt(N);
  for (size_t i = 0; i < N; ++i) ft[i] = (T)f[i];
  const T L[2] = {(T)len_xy[0], (T)len_xy[1]};
  int rc = poisson_solve<T>(nu, L, bc, zg, ft.data(), pt.data(), nthreads, (T)shift);
  for (size_t i = 0; i < N; ++i) p[i] = (double)pt[i];
  return rc;
}

template <typename T>
int apply_t(const int n[3], const double len_xy[2], const int bc[3], const double* dzf, const double* p, double* out,
            int nthreads, double shift = 0, int faces = 0) {
  ZGrid<T> zg(n[2], bc[2], dzf, faces != 0);
  const int nu[3] = {n[0], n[1], zg.nz};
  const size_t N = (size_t)n[0] * n[1] * zg.nz;
  std::vector<T> pt(N), ot(N);
  for (size_t i = 0; i < N; ++i) pt[i] = (T)p[i];
  const T L[2] = {(T)len_xy[0], (T)len_xy[1]};
  apply_laplacian<T>(nu, L, bc, zg, pt.data(), ot.data(), nthreads, (T)shift);
  for (size_t i = 0; i < N; ++i) out[i] = (double)ot[i];
  return 0;
}

int nthreads_or_default(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

}  // namespace

extern "C" {

// prec_bits: 64 = double, 80 = long double, 128 = __float128.  Inputs and outputs are double;
// the arithmetic runs in the requested precision.  Returns 0 on success, <0 on bad arguments.
int oracle_poisson_solve(int prec_bits, const int n[3], const double len_xy[2], const int bc[3], const double* dzf,
                         const double* f, double* p, int nthreads) {
  int rc = check_args(n, bc, dzf);
  if (rc) return rc;
  nthreads = nthreads_or_default(nthreads);
  if (prec_bits == 64) return solve_t<double>(n, len_xy, bc, dzf, f, p, nthreads);
  if (prec_bits == 80) return solve_t<long double>(n, len_xy, bc, dzf, f, p, nthreads);
  if (prec_bits == 128) return solve_t<quad>(n, len_xy, bc, dzf, f, p, nthreads);
  return -1;
}

// out = L_h p (eq. poi, non-uniform z as in the Validation section).
int oracle_apply_laplacian(int prec_bits, const int n[3], const double len_xy[2], const int bc[3],
                           const double* dzf, const double* p, double* out, int nthreads) {
  int rc = check_args(n, bc, dzf);
  if (rc) return rc;
  nthreads = nthreads_or_default(nthreads);
  if (prec_bits == 64) return apply_t<double>(n, len_xy, bc, dzf, p, out, nthreads);
  if (prec_bits == 80) return apply_t<long double>(n, len_xy, bc, dzf, p, out, nthreads);
  if (prec_bits == 128) return apply_t<quad>(n, len_xy, bc, dzf, p, out, nthreads);
  return -1;
}

// (L_h + shift) p = f (Eq. up_id_2 in Helmholtz form) and its operator, on the cell grid (faces = 0)
// or on the interior z-faces of the dzf cells (faces = 1, Dirichlet walls only: w = 0 on the wall
// faces).  n[2] counts the dzf cells; f, p, out hold n[0] n[1] (n[2] - faces) values.
int oracle_helmholtz_solve(int prec_bits, const int n[3], const double len_xy[2], const int bc[3], const double* dzf,
                           double shift, int faces, const double* f, double* p, int nthreads) {
  int rc = check_args(n, bc, dzf);
  if (rc) return rc;
  if (faces && (bc[2] != BC_DD || n[2] < 2)) return -1;
  nthreads = nthreads_or_default(nthreads);
  if (prec_bits == 64) return solve_t<double>(n, len_xy, bc, dzf, f, p, nthreads, shift, faces);
  if (prec_bits == 80) return solve_t<long double>(n, len_xy, bc, dzf, f, p, nthreads, shift, faces);
  if (prec_bits == 128) return solve_t<quad>(n, len_xy, bc, dzf, f, p, nthreads, shift, faces);
  return -1;
}

int oracle_apply_helmholtz(int prec_bits, const int n[3], const double len_xy[2], const int bc[3], const double* dzf,
                           double shift, int faces, const double* p, double* out, int nthreads) {
  int rc = check_args(n, bc, dzf);
  if (rc) return rc;
  if (faces && (bc[2] != BC_DD || n[2] < 2)) return -1;
  nthreads = nthreads_or_default(nthreads);
  if (prec_bits == 64) return apply_t<double>(n, len_xy, bc, dzf, p, out, nthreads, shift, faces);
  if (prec_bits == 80) return apply_t<long double>(n, len_xy, bc, dzf, p, out, nthreads, shift, faces);
  if (prec_bits == 128) return apply_t<quad>(n, len_xy, bc, dzf, p, out, nthreads, shift, faces);
  return -1;
}

// Dense orthonormal eigenbasis E (row-major n x n, columns = eigenvectors) and unit-spacing
// eigenvalues lam of the 1-D operator with boundary condition bc.
int oracle_eigenbasis(int bc, int n, double* E, double* lam) {
  if (n < 1 || bc < 0 || bc > 4) return -1;
  std::vector<double> e, l;
  eigenbasis<double>(bc, n, e, l);
  std::memcpy(E, e.data(), sizeof(double) * e.size());
  std::memcpy(lam, l.data(), sizeof(double) * l.size());
  return 0;
}

// Rows of the z operator for one mode: a_k p_{k-1} + b_k p_k + c_k p_{k+1}; a_0 = c_{nz-1} = 0 at walls.
int oracle_z_rows(int bc_z, int nz, const double* dzf, double* a, double* b, double* c) {
  if (nz < 1 || bc_z < 0 || bc_z > 4) return -1;
  ZGrid<double> zg(nz, bc_z, dzf);
  std::vector<double> va, vb, vc;
  z_rows<double>(zg, va, vb, vc);
  for (int k = 0; k < nz; ++k) {
    a[k] = va[k];
    b[k] = vb[k];
    c[k] = vc[k];
  }
  return 0;
}

// Plain Thomas solve (no pivoting) of one tridiagonal system.
int oracle_thomas(int n, const double* a, const double* b, const double* c, const double* d, double* x) {
  if (n < 1) return -1;
  thomas<double>(n, a, b, c, d, x);
  return 0;
}

void oracle_set_fault(int mode) { g_fault = mode; }

}  // extern "C"

// =================================================================================================
// Fractional-step pieces around the Poisson solve (Numerical method: Eq. up, Eq. poi_ns and the
// correction and pressure update after it; Eq. dt and its chkdt listing), for a channel: x and y
// periodic, no-slip / no-penetration walls at z = 0 and z = Lz, Neumann pressure at the walls.
//
// Staggered (marker-and-cell) arrays, all Nx x Ny x Nz, x fastest:
//   u[k][j][i] on the x-face between cells i and i+1, v on the y-face between j and j+1,
//   w on the z-face between k and k+1 (w[Nz-1] is the top wall and stays 0; the bottom wall w = 0
//   sits below k = 0), p at cell centres.
// Advection is the conservative divergence of u (x) u with arithmetic two-point averages; diffusion
// is the same 3-point Laplacian as the pressure with no-slip ghosts (ghost = -interior at the wall).
// All loops are plain double arithmetic.
// =================================================================================================
namespace {

struct Chan {
  int nx, ny, nz;
  double dx, dy;
  std::vector<double> dzf, dzc;  // dzc[k] = distance between centres k-1 and k (k = 0..nz), wall ghosts
  Chan(const int n[3], const double len_xy[2], const double* dz) : nx(n[0]), ny(n[1]), nz(n[2]), dzf(n[2]), dzc(n[2] + 1) {
    dx = len_xy[0] / nx;
    dy = len_xy[1] / ny;
    for (int k = 0; k < nz; ++k) dzf[k] = dz[k];
    for (int k = 1; k < nz; ++k) dzc[k] = 0.5 * (dzf[k - 1] + dzf[k]);
    dzc[0] = dzf[0];
    dzc[nz] = dzf[nz - 1];
  }
  size_t id(int i, int j, int k) const {
    i = (i % nx + nx) % nx;
    j = (j % ny + ny) % ny;
    return (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * k);
  }
  size_t size() const { return (size_t)nx * ny * nz; }
};

// cell-centred value of a face field with the wall rules: u, v (tangential) have ghosts -u at the
// walls; w is zero on both walls.
inline double U(const Chan& g, const double* a, int i, int j, int k) {
  if (k < 0) return -a[g.id(i, j, 0)];
  if (k >= g.nz) return -a[g.id(i, j, g.nz - 1)];
  return a[g.id(i, j, k)];
}
inline double W(const Chan& g, const double* w, int i, int j, int k) {
  if (k < 0 || k >= g.nz - 1) return 0.0;
  return w[g.id(i, j, k)];
}

void divergence(const Chan& g, const double* u, const double* v, const double* w, double* out) {
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i)
        out[g.id(i, j, k)] = (u[g.id(i, j, k)] - u[g.id(i - 1, j, k)]) / g.dx +
                             (v[g.id(i, j, k)] - v[g.id(i, j - 1, k)]) / g.dy +
                             (W(g, w, i, j, k) - W(g, w, i, j, k - 1)) / g.dzf[k];
}

void gradient(const Chan& g, const double* q, double* gx, double* gy, double* gz) {
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const size_t c = g.id(i, j, k);
        gx[c] = (q[g.id(i + 1, j, k)] - q[c]) / g.dx;
        gy[c] = (q[g.id(i, j + 1, k)] - q[c]) / g.dy;
        gz[c] = (k < g.nz - 1) ? (q[g.id(i, j, k + 1)] - q[c]) / g.dzc[k + 1] : 0.0;
      }
}

// 3-point Laplacian of a tangential velocity (no-slip ghosts) at its own location
double lap_t(const Chan& g, const double* a, int i, int j, int k) {
  const double c = a[g.id(i, j, k)];
  const double lx = (a[g.id(i - 1, j, k)] - 2 * c + a[g.id(i + 1, j, k)]) / (g.dx * g.dx);
  const double ly = (a[g.id(i, j - 1, k)] - 2 * c + a[g.id(i, j + 1, k)]) / (g.dy * g.dy);
  const double lz = ((U(g, a, i, j, k + 1) - c) / g.dzc[k + 1] - (c - U(g, a, i, j, k - 1)) / g.dzc[k]) / g.dzf[k];
  return lx + ly + lz;
}

// momentum right-hand side A(u) + nu L(u) of Eq. up (advection as -div(u u))
void momentum_rhs(const Chan& g, double nu, const double* u, const double* v, const double* w, double* ru,
                  double* rv, double* rw) {
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const size_t c = g.id(i, j, k);
        // u on the face (i+1/2, j, k)
        {
          const double ue = 0.5 * (u[c] + u[g.id(i + 1, j, k)]), uw = 0.5 * (u[g.id(i - 1, j, k)] + u[c]);
          const double un = 0.5 * (u[c] + u[g.id(i, j + 1, k)]) * 0.5 * (v[c] + v[g.id(i + 1, j, k)]);
          const double us = 0.5 * (u[g.id(i, j - 1, k)] + u[c]) * 0.5 * (v[g.id(i, j - 1, k)] + v[g.id(i + 1, j - 1, k)]);
          const double ut = 0.5 * (u[c] + U(g, u, i, j, k + 1)) * 0.5 * (W(g, w, i, j, k) + W(g, w, i + 1, j, k));
          const double ub = 0.5 * (U(g, u, i, j, k - 1) + u[c]) * 0.5 * (W(g, w, i, j, k - 1) + W(g, w, i + 1, j, k - 1));
          // planted 4: the u z-flux divided by the centre distance instead of the cell width
          const double hz = (g_fault == 4) ? g.dzc[k + 1] : g.dzf[k];
          const double adv = (ue * ue - uw * uw) / g.dx + (un - us) / g.dy + (ut - ub) / hz;
          ru[c] = -adv + nu * lap_t(g, u, i, j, k);
        }
        // v on the face (i, j+1/2, k)
        {
          const double ve = 0.5 * (v[c] + v[g.id(i + 1, j, k)]) * 0.5 * (u[c] + u[g.id(i, j + 1, k)]);
          const double vw = 0.5 * (v[g.id(i - 1, j, k)] + v[c]) * 0.5 * (u[g.id(i - 1, j, k)] + u[g.id(i - 1, j + 1, k)]);
          const double vn = 0.5 * (v[c] + v[g.id(i, j + 1, k)]), vs = 0.5 * (v[g.id(i, j - 1, k)] + v[c]);
          const double vt = 0.5 * (v[c] + U(g, v, i, j, k + 1)) * 0.5 * (W(g, w, i, j, k) + W(g, w, i, j + 1, k));
          const double vb = 0.5 * (U(g, v, i, j, k - 1) + v[c]) * 0.5 * (W(g, w, i, j, k - 1) + W(g, w, i, j + 1, k - 1));
          const double adv = (ve - vw) / g.dx + (vn * vn - vs * vs) / g.dy + (vt - vb) / g.dzf[k];
          rv[c] = -adv + nu * lap_t(g, v, i, j, k);
        }
        // w on the face (i, j, k+1/2); the top wall face stays at rest
        if (k == g.nz - 1) {
          rw[c] = 0.0;
        } else {
          const double wc = w[c];
          const double we = 0.5 * (wc + W(g, w, i + 1, j, k)) * 0.5 * (u[c] + u[g.id(i, j, k + 1)]);
          const double ww = 0.5 * (W(g, w, i - 1, j, k) + wc) * 0.5 * (u[g.id(i - 1, j, k)] + u[g.id(i - 1, j, k + 1)]);
          const double wn = 0.5 * (wc + W(g, w, i, j + 1, k)) * 0.5 * (v[c] + v[g.id(i, j, k + 1)]);
          const double ws = 0.5 * (W(g, w, i, j - 1, k) + wc) * 0.5 * (v[g.id(i, j - 1, k)] + v[g.id(i, j - 1, k + 1)]);
          const double wt = 0.5 * (wc + W(g, w, i, j, k + 1)), wb = 0.5 * (W(g, w, i, j, k - 1) + wc);
          // planted 5: the w z-flux divided by the cell width instead of the centre distance
          const double hz = (g_fault == 5) ? g.dzf[k] : g.dzc[k + 1];
          const double adv = (we - ww) / g.dx + (wn - ws) / g.dy + (wt * wt - wb * wb) / hz;
          const double lx = (W(g, w, i - 1, j, k) - 2 * wc + W(g, w, i + 1, j, k)) / (g.dx * g.dx);
          const double ly = (W(g, w, i, j - 1, k) - 2 * wc + W(g, w, i, j + 1, k)) / (g.dy * g.dy);
          const double lz = ((W(g, w, i, j, k + 1) - wc) / g.dzf[k + 1] - (wc - W(g, w, i, j, k - 1)) / g.dzf[k]) / g.dzc[k + 1];
          rw[c] = -adv + nu * (lx + ly + lz);
        }
      }
}

// largest inverse advective time scale (chkdt listing; the y and z rows follow the x row by symmetry)
double max_dti(const Chan& g, const double* u, const double* v, const double* w) {
  double dti = 0;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const size_t c = g.id(i, j, k);
        const double ux = std::fabs(u[c]);
        const double vx = 0.25 * std::fabs(v[c] + v[g.id(i, j - 1, k)] + v[g.id(i + 1, j, k)] + v[g.id(i + 1, j - 1, k)]);
        const int kb = (g_fault == 7) ? k + 1 : k - 1;  // planted 7: the wrong pair of w faces
        const double wx = 0.25 * std::fabs(W(g, w, i, j, k) + W(g, w, i, j, kb) + W(g, w, i + 1, j, k) + W(g, w, i + 1, j, kb));
        const double dtix = ux / g.dx + vx / g.dy + wx / g.dzf[k];
        const double uy = 0.25 * std::fabs(u[c] + u[g.id(i - 1, j, k)] + u[g.id(i, j + 1, k)] + u[g.id(i - 1, j + 1, k)]);
        const double vy = std::fabs(v[c]);
        const double wy = 0.25 * std::fabs(W(g, w, i, j, k) + W(g, w, i, j, k - 1) + W(g, w, i, j + 1, k) + W(g, w, i, j + 1, k - 1));
        const double dtiy = uy / g.dx + vy / ((g_fault == 8) ? g.dx : g.dy) + wy / g.dzf[k];  // planted 8: x spacing
        const double uz = 0.25 * std::fabs(u[c] + u[g.id(i - 1, j, k)] + U(g, u, i, j, k + 1) + U(g, u, i - 1, j, k + 1));
        const double vz = 0.25 * std::fabs(v[c] + v[g.id(i, j - 1, k)] + U(g, v, i, j, k + 1) + U(g, v, i, j - 1, k + 1));
        const double wz = std::fabs(W(g, w, i, j, k));
        const double dtiz = uz / g.dx + vz / g.dy + wz / ((g_fault == 6) ? g.dzf[k] : g.dzc[k + 1]);  // planted 6: cell width
        dti = std::max(dti, std::max(dtix, std::max(dtiy, dtiz)));
      }
  return dti;
}

// dt = cfl * min(sqrt(3)/dti, 1.65 dl^2/nu), dl = min(dx, dy, min dzf) (Eq. dt)
double stable_dt(const Chan& g, double nu, double cfl, const double* u, const double* v, const double* w) {
  double dl = std::min(g.dx, g.dy);
  for (int k = 0; k < g.nz; ++k) dl = std::min(dl, g.dzf[k]);
  const double dti = max_dti(g, u, v, w);
  double dt = 1.65 * dl * dl / nu;
  if (dti > 0) dt = std::min(dt, std::sqrt(3.0) / dti);
  return cfl * dt;
}

double bulk_u(const Chan& g, const double* u) {
  double s = 0, wsum = 0;
  for (int k = 0; k < g.nz; ++k) {
    double pl = 0;
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) pl += u[g.id(i, j, k)];
    s += g.dzf[k] * pl;
    wsum += g.dzf[k];
  }
  return s / (wsum * g.nx * g.ny);
}

const double RK_A[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
const double RK_B[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};

// The viscous operator L of the momentum equations alone: lap_t for u and v (no-slip ghosts), the
// face-grid second difference for w (zero on both walls; the top wall face stays 0).
void velocity_laplacian(const Chan& g, const double* u, const double* v, const double* w, double* lu, double* lv,
                        double* lw) {
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const size_t c = g.id(i, j, k);
        lu[c] = lap_t(g, u, i, j, k);
        lv[c] = lap_t(g, v, i, j, k);
        if (k == g.nz - 1) {
          lw[c] = 0.0;
          continue;
        }
        const double wc = w[c];
        const double lx = (W(g, w, i - 1, j, k) - 2 * wc + W(g, w, i + 1, j, k)) / (g.dx * g.dx);
        const double ly = (W(g, w, i, j - 1, k) - 2 * wc + W(g, w, i, j + 1, k)) / (g.dy * g.dy);
        const double lz = ((W(g, w, i, j, k + 1) - wc) / g.dzf[k + 1] - (wc - W(g, w, i, j, k - 1)) / g.dzf[k]) / g.dzc[k + 1];
        lw[c] = lx + ly + lz;
      }
}

}  // namespace

extern "C" {

int oracle_divergence(const int n[3], const double len_xy[2], const double* dzf, const double* u, const double* v,
                      const double* w, double* out) {
  Chan g(n, len_xy, dzf);
  divergence(g, u, v, w, out);
  return 0;
}

int oracle_gradient(const int n[3], const double len_xy[2], const double* dzf, const double* q, double* gx, double* gy,
                    double* gz) {
  Chan g(n, len_xy, dzf);
  gradient(g, q, gx, gy, gz);
  return 0;
}

int oracle_momentum_rhs(const int n[3], const double len_xy[2], const double* dzf, double nu, const double* u,
                        const double* v, const double* w, double* ru, double* rv, double* rw) {
  Chan g(n, len_xy, dzf);
  momentum_rhs(g, nu, u, v, w, ru, rv, rw);
  return 0;
}

double oracle_stable_dt(const int n[3], const double len_xy[2], const double* dzf, double nu, double cfl,
                        const double* u, const double* v, const double* w) {
  Chan g(n, len_xy, dzf);
  return stable_dt(g, nu, cfl, u, v, w);
}

// Projection of a face field on discretely divergence-free fields: u - G L^-1 D u (the correction of
// the fractional step with the gamma dt factors cancelled).  Pressure problem: (P, P, NN).
int oracle_project(const int n[3], const double len_xy[2], const double* dzf, const double* u, const double* v,
                   const double* w, double* uo, double* vo, double* wo, double* phi_out, int nthreads) {
  Chan g(n, len_xy, dzf);
  const size_t N = g.size();
  std::vector<double> d(N), phi(N), gx(N), gy(N), gz(N);
  divergence(g, u, v, w, d.data());
  const int bc[3] = {BC_P, BC_P, BC_NN};
  int rc = solve_t<double>(n, len_xy, bc, dzf, d.data(), phi.data(), nthreads_or_default(nthreads));
  if (rc) return rc;
  gradient(g, phi.data(), gx.data(), gy.data(), gz.data());
  for (size_t c = 0; c < N; ++c) {
    uo[c] = u[c] - gx[c];
    vo[c] = v[c] - gy[c];
    wo[c] = w[c] - gz[c];
  }
  if (phi_out) std::memcpy(phi_out, phi.data(), N * sizeof(double));
  return 0;
}

// One explicit low-storage RK3 step (Eq. up with alpha, beta, gamma = alpha + beta), in place on
// u, v, w, p.  dt is computed from the state at the start of the step (Eq. dt with cfl) unless
// dt_in > 0.  After each substage's correction u is shifted to bulk velocity ubulk (constant flow
// rate).  Returns the dt used through *dt_out.
int oracle_rk3_step(const int n[3], const double len_xy[2], const double* dzf, double nu, double cfl, double ubulk,
                    double dt_in, double* u, double* v, double* w, double* p, double* dt_out, int nthreads) {
  Chan g(n, len_xy, dzf);
  const size_t N = g.size();
  const double dt = (dt_in > 0) ? dt_in : stable_dt(g, nu, cfl, u, v, w);
  std::vector<double> ru(N), rv(N), rw(N), pu(N, 0.0), pv(N, 0.0), pw(N, 0.0), gx(N), gy(N), gz(N), d(N), phi(N);
  const int bc[3] = {BC_P, BC_P, BC_NN};
  nthreads = nthreads_or_default(nthreads);
  for (int s = 0; s < 3; ++s) {
    const double a = RK_A[s], b = RK_B[s], gm = a + b;
    momentum_rhs(g, nu, u, v, w, ru.data(), rv.data(), rw.data());
    gradient(g, p, gx.data(), gy.data(), gz.data());
    for (size_t c = 0; c < N; ++c) {
      u[c] += dt * (a * ru[c] + b * pu[c] - gm * gx[c]);
      v[c] += dt * (a * rv[c] + b * pv[c] - gm * gy[c]);
      w[c] += dt * (a * rw[c] + b * pw[c] - gm * gz[c]);
    }
    divergence(g, u, v, w, d.data());
    for (size_t c = 0; c < N; ++c) d[c] /= gm * dt;
    int rc = solve_t<double>(n, len_xy, bc, dzf, d.data(), phi.data(), nthreads);
    if (rc) return rc;
    gradient(g, phi.data(), gx.data(), gy.data(), gz.data());
    for (size_t c = 0; c < N; ++c) {
      u[c] -= gm * dt * gx[c];
      v[c] -= gm * dt * gy[c];
      w[c] -= gm * dt * gz[c];
      p[c] += phi[c];
    }
    const double shift = ubulk - bulk_u(g, u);
    for (size_t c = 0; c < N; ++c) u[c] += shift;
    pu.swap(ru);
    pv.swap(rv);
    pw.swap(rw);
  }
  if (dt_out) *dt_out = dt;
  return 0;
}

// One RK3 step with implicit (Crank-Nicolson) viscous diffusion, the second form of the Numerical
// method: per substage
//   u** = u^k + dt (alpha A u^k + beta A u^{k-1} + gamma (-G p + nu L u^k))            (Eq. up_id)
//   u* - gamma nu dt/2 L u* = u** - gamma nu dt/2 L u^k                                (Eq. up_id_2)
//   L Phi = D u* / (gamma dt),  u^{k+1} = u* - gamma dt G Phi,
//   p^{k+1/2} = p^{k-1/2} + Phi - gamma nu dt/2 L Phi,
// A the advection alone.  Eq. up_id_2 is solved per component as the Helmholtz problem
// (L + s) u* = s rhs with s = -2/(gamma nu dt): u and v on the cell grid with no-slip ghosts (x, y
// periodic, z Dirichlet), w on the interior z-faces.  The pressure Laplacian of Phi has the Neumann
// walls of the pressure.  dt as oracle_rk3_step; forcing shifts u to ubulk when forcing != 0.
int oracle_rk3_step_implicit(const int n[3], const double len_xy[2], const double* dzf, double nu, double cfl,
                             double ubulk, int forcing, double dt_in, double* u, double* v, double* w, double* p,
                             double* dt_out, int nthreads) {
  Chan g(n, len_xy, dzf);
  const size_t N = g.size();
  const size_t NW = (size_t)g.nx * g.ny * (g.nz - 1);  // interior z-faces
  const double dt = (dt_in > 0) ? dt_in : stable_dt(g, nu, cfl, u, v, w);
  std::vector<double> au(N), av(N), aw(N), pu(N, 0.0), pv(N, 0.0), pw(N, 0.0), lu(N), lv(N), lw(N);
  std::vector<double> gx(N), gy(N), gz(N), d(N), phi(N), lphi(N), ru(N), rv(N), rw(N), z0(N, 0.0);
  const int bcp[3] = {BC_P, BC_P, BC_NN};
  const int bcv[3] = {BC_P, BC_P, BC_DD};
  nthreads = nthreads_or_default(nthreads);
  for (int s = 0; s < 3; ++s) {
    const double a = RK_A[s], b = RK_B[s], gm = a + b;
    const double h = gm * nu * dt / 2, sh = -1.0 / h;
    momentum_rhs(g, 0.0, u, v, w, au.data(), av.data(), aw.data());  // advection only
    velocity_laplacian(g, u, v, w, lu.data(), lv.data(), lw.data());
    gradient(g, p, gx.data(), gy.data(), gz.data());
    for (size_t c = 0; c < N; ++c) {
      const double uss = u[c] + dt * (a * au[c] + b * pu[c] + gm * (-gx[c] + nu * lu[c]));
      const double vss = v[c] + dt * (a * av[c] + b * pv[c] + gm * (-gy[c] + nu * lv[c]));
      const double wss = w[c] + dt * (a * aw[c] + b * pw[c] + gm * (-gz[c] + nu * lw[c]));
      ru[c] = sh * (uss - h * lu[c]);
      rv[c] = sh * (vss - h * lv[c]);
      rw[c] = sh * (wss - h * lw[c]);
    }
    int rc = solve_t<double>(n, len_xy, bcv, dzf, ru.data(), u, nthreads, sh, 0);
    if (rc) return rc;
    rc = solve_t<double>(n, len_xy, bcv, dzf, rv.data(), v, nthreads, sh, 0);
    if (rc) return rc;
    rc = solve_t<double>(n, len_xy, bcv, dzf, rw.data(), w, nthreads, sh, 1);  // the first Nz-1 planes
    if (rc) return rc;
    for (size_t c = NW; c < N; ++c) w[c] = 0.0;  // top wall face
    divergence(g, u, v, w, d.data());
    for (size_t c = 0; c < N; ++c) d[c] /= gm * dt;
    rc = solve_t<double>(n, len_xy, bcp, dzf, d.data(), phi.data(), nthreads);
    if (rc) return rc;
    gradient(g, phi.data(), gx.data(), gy.data(), gz.data());
    rc = apply_t<double>(n, len_xy, bcp, dzf, phi.data(), lphi.data(), nthreads);
    if (rc) return rc;
    for (size_t c = 0; c < N; ++c) {
      u[c] -= gm * dt * gx[c];
      v[c] -= gm * dt * gy[c];
      w[c] -= gm * dt * gz[c];
      p[c] += phi[c] - h * lphi[c];
    }
    if (forcing) {
      const double shift = ubulk - bulk_u(g, u);
      for (size_t c = 0; c < N; ++c) u[c] += shift;
    }
    pu.swap(au);
    pv.swap(av);
    pw.swap(aw);
  }
  if (dt_out) *dt_out = dt;
  return 0;
}

}  // extern "C"

// =================================================================================================
// The same fractional step in a box whose every direction is either periodic or bounded by no-slip
// walls, with an optional moving lid (the top z wall moving with velocity lid along x): the flows the
// paper lists for its solver -- lid-driven cavity (walls everywhere), square duct (x periodic),
// channel (z walls), decaying Taylor-Green vortex (periodic everywhere).  Written separately from
// the channel code above from the same marker-and-cell definitions, so that the two cross-check:
//   * a velocity component normal to a walled direction lives on that direction's faces and is zero
//     on both wall faces (the high wall face is its last stored face);
//   * a tangential component beyond a wall takes the ghost 2 U_wall - (value at the wall cell), with
//     U_wall = lid for u at the top z wall and 0 otherwise;
//   * the pressure is Neumann at walls, periodic elsewhere.
// =================================================================================================
namespace {

struct Box {
  int n[3];
  bool wall[3];
  double lid;
  double dx, dy;
  std::vector<double> dzf, dzc;  // dzc[k]: centre distance between k-1 and k, k = 0..nz (wall ghosts: dzf)
  Box(const int n_[3], const int wall_[3], double lid_, const double len_xy[2], const double* dz)
      : lid(lid_), dzf(n_[2]), dzc(n_[2] + 1) {
    for (int d = 0; d < 3; ++d) {
      n[d] = n_[d];
      wall[d] = wall_[d] != 0;
    }
    dx = len_xy[0] / n[0];
    dy = len_xy[1] / n[1];
    const int nz = n[2];
    for (int k = 0; k < nz; ++k) dzf[k] = dz[k];
    for (int k = 1; k < nz; ++k) dzc[k] = 0.5 * (dzf[k - 1] + dzf[k]);
    dzc[0] = wall[2] ? dzf[0] : 0.5 * (dzf[nz - 1] + dzf[0]);
    dzc[nz] = wall[2] ? dzf[nz - 1] : dzc[0];
  }
  size_t size() const { return (size_t)n[0] * n[1] * n[2]; }
  size_t at(int i, int j, int k) const { return (size_t)i + (size_t)n[0] * ((size_t)j + (size_t)n[1] * k); }
  // component c (0 u, 1 v, 2 w) of face field a at (i, j, k), each index at most one cell outside
  double V(const double* a, int c, int i, int j, int k) const {
    int id[3] = {i, j, k};
    double sgn = 1.0, add = 0.0;
    for (int d = 0; d < 3; ++d) {
      int& x = id[d];
      if (wall[d] && d == c && (x < 0 || x >= n[d] - 1)) return 0.0;  // normal velocity at / beyond a wall
      if (x >= 0 && x < n[d]) continue;
      if (!wall[d]) {
        x = (x + n[d]) % n[d];
        continue;
      }
      // crossing a wall maps the value v to 2 U_wall - v (a corner ghost crosses two walls, x first)
      const bool high = x >= n[d];
      x = high ? n[d] - 1 : 0;
      add = -add + ((high && d == 2 && c == 0) ? 2.0 * lid : 0.0);
      sgn = -sgn;
    }
    return sgn * a[at(id[0], id[1], id[2])] + add;
  }
  double P(const double* q, int i, int j, int k) const {  // pressure-like cell field, Neumann at walls
    int id[3] = {i, j, k};
    for (int d = 0; d < 3; ++d) {
      int& x = id[d];
      if (x >= 0 && x < n[d]) continue;
      x = wall[d] ? (x < 0 ? 0 : n[d] - 1) : (x + n[d]) % n[d];
    }
    return q[at(id[0], id[1], id[2])];
  }
  bool wall_face(int c, int i, int j, int k) const {
    const int x = (c == 0) ? i : (c == 1 ? j : k);
    return wall[c] && x == n[c] - 1;
  }
};

void box_divergence(const Box& g, const double* u, const double* v, const double* w, double* out) {
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i)
        out[g.at(i, j, k)] = (g.V(u, 0, i, j, k) - g.V(u, 0, i - 1, j, k)) / g.dx +
                             (g.V(v, 1, i, j, k) - g.V(v, 1, i, j - 1, k)) / g.dy +
                             (g.V(w, 2, i, j, k) - g.V(w, 2, i, j, k - 1)) / g.dzf[k];
}

void box_gradient(const Box& g, const double* q, double* gx, double* gy, double* gz) {
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        const size_t c = g.at(i, j, k);
        const double qc = q[c];
        gx[c] = g.wall_face(0, i, j, k) ? 0.0 : (g.P(q, i + 1, j, k) - qc) / g.dx;
        gy[c] = g.wall_face(1, i, j, k) ? 0.0 : (g.P(q, i, j + 1, k) - qc) / g.dy;
        gz[c] = g.wall_face(2, i, j, k) ? 0.0 : (g.P(q, i, j, k + 1) - qc) / g.dzc[k + 1];
      }
}

// viscous operator of each component at its own faces (3-point differences; z metrics of cell
// centres for u, v and of faces for w)
void box_laplacian(const Box& g, const double* u, const double* v, const double* w, double* lu, double* lv,
                   double* lw) {
  const double idx2 = 1.0 / (g.dx * g.dx), idy2 = 1.0 / (g.dy * g.dy);
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        const size_t c = g.at(i, j, k);
        const double* F[3] = {u, v, w};
        double* L[3] = {lu, lv, lw};
        for (int q = 0; q < 3; ++q) {
          if (g.wall_face(q, i, j, k)) {
            L[q][c] = 0.0;
            continue;
          }
          const double* a = F[q];
          const double ac = g.V(a, q, i, j, k);
          const double lx = (g.V(a, q, i - 1, j, k) - 2 * ac + g.V(a, q, i + 1, j, k)) * idx2;
          const double ly = (g.V(a, q, i, j - 1, k) - 2 * ac + g.V(a, q, i, j + 1, k)) * idy2;
          double lz;
          if (q < 2) {
            lz = ((g.V(a, q, i, j, k + 1) - ac) / g.dzc[k + 1] - (ac - g.V(a, q, i, j, k - 1)) / g.dzc[k]) / g.dzf[k];
          } else {
            const double dzu = g.dzf[(k + 1) % g.n[2]], mid = g.dzc[k + 1];
            lz = ((g.V(a, q, i, j, k + 1) - ac) / dzu - (ac - g.V(a, q, i, j, k - 1)) / g.dzf[k]) / mid;
          }
          L[q][c] = lx + ly + lz;
        }
      }
}

// conservative advection -div(u u) with two-point averages at each component's faces
void box_advection(const Box& g, const double* u, const double* v, const double* w, double* au, double* av,
                   double* aw) {
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        const size_t c = g.at(i, j, k);
        auto U = [&](int a, int b, int e) { return g.V(u, 0, a, b, e); };
        auto Vv = [&](int a, int b, int e) { return g.V(v, 1, a, b, e); };
        auto Ww = [&](int a, int b, int e) { return g.V(w, 2, a, b, e); };
        if (g.wall_face(0, i, j, k)) {
          au[c] = 0.0;
        } else {  // u at (i+1/2, j, k)
          const double ue = 0.5 * (U(i, j, k) + U(i + 1, j, k)), uw = 0.5 * (U(i - 1, j, k) + U(i, j, k));
          const double un = 0.5 * (U(i, j, k) + U(i, j + 1, k)) * 0.5 * (Vv(i, j, k) + Vv(i + 1, j, k));
          const double us = 0.5 * (U(i, j - 1, k) + U(i, j, k)) * 0.5 * (Vv(i, j - 1, k) + Vv(i + 1, j - 1, k));
          const double ut = 0.5 * (U(i, j, k) + U(i, j, k + 1)) * 0.5 * (Ww(i, j, k) + Ww(i + 1, j, k));
          const double ub = 0.5 * (U(i, j, k - 1) + U(i, j, k)) * 0.5 * (Ww(i, j, k - 1) + Ww(i + 1, j, k - 1));
          au[c] = -((ue * ue - uw * uw) / g.dx + (un - us) / g.dy + (ut - ub) / g.dzf[k]);
        }
        if (g.wall_face(1, i, j, k)) {
          av[c] = 0.0;
        } else {  // v at (i, j+1/2, k)
          const double ve = 0.5 * (Vv(i, j, k) + Vv(i + 1, j, k)) * 0.5 * (U(i, j, k) + U(i, j + 1, k));
          const double vw = 0.5 * (Vv(i - 1, j, k) + Vv(i, j, k)) * 0.5 * (U(i - 1, j, k) + U(i - 1, j + 1, k));
          const double vn = 0.5 * (Vv(i, j, k) + Vv(i, j + 1, k)), vs = 0.5 * (Vv(i, j - 1, k) + Vv(i, j, k));
          const double vt = 0.5 * (Vv(i, j, k) + Vv(i, j, k + 1)) * 0.5 * (Ww(i, j, k) + Ww(i, j + 1, k));
          const double vb = 0.5 * (Vv(i, j, k - 1) + Vv(i, j, k)) * 0.5 * (Ww(i, j, k - 1) + Ww(i, j + 1, k - 1));
          av[c] = -((ve - vw) / g.dx + (vn * vn - vs * vs) / g.dy + (vt - vb) / g.dzf[k]);
        }
        if (g.wall_face(2, i, j, k)) {
          aw[c] = 0.0;
        } else {  // w at (i, j, k+1/2)
          const double we = 0.5 * (Ww(i, j, k) + Ww(i + 1, j, k)) * 0.5 * (U(i, j, k) + U(i, j, k + 1));
          const double ww = 0.5 * (Ww(i - 1, j, k) + Ww(i, j, k)) * 0.5 * (U(i - 1, j, k) + U(i - 1, j, k + 1));
          const double wn = 0.5 * (Ww(i, j, k) + Ww(i, j + 1, k)) * 0.5 * (Vv(i, j, k) + Vv(i, j, k + 1));
          const double ws = 0.5 * (Ww(i, j - 1, k) + Ww(i, j, k)) * 0.5 * (Vv(i, j - 1, k) + Vv(i, j - 1, k + 1));
          const double wt = 0.5 * (Ww(i, j, k) + Ww(i, j, k + 1)), wb = 0.5 * (Ww(i, j, k - 1) + Ww(i, j, k));
          aw[c] = -((we - ww) / g.dx + (wn - ws) / g.dy + (wt * wt - wb * wb) / g.dzc[k + 1]);
        }
      }
}

double box_max_dti(const Box& g, const double* u, const double* v, const double* w) {
  double dti = 0;
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        auto U = [&](int a, int b, int e) { return g.V(u, 0, a, b, e); };
        auto Vv = [&](int a, int b, int e) { return g.V(v, 1, a, b, e); };
        auto Ww = [&](int a, int b, int e) { return g.V(w, 2, a, b, e); };
        const double dtix = std::fabs(U(i, j, k)) / g.dx +
                            0.25 * std::fabs(Vv(i, j, k) + Vv(i, j - 1, k) + Vv(i + 1, j, k) + Vv(i + 1, j - 1, k)) / g.dy +
                            0.25 * std::fabs(Ww(i, j, k) + Ww(i, j, k - 1) + Ww(i + 1, j, k) + Ww(i + 1, j, k - 1)) / g.dzf[k];
        const double dtiy = 0.25 * std::fabs(U(i, j, k) + U(i - 1, j, k) + U(i, j + 1, k) + U(i - 1, j + 1, k)) / g.dx +
                            std::fabs(Vv(i, j, k)) / g.dy +
                            0.25 * std::fabs(Ww(i, j, k) + Ww(i, j, k - 1) + Ww(i, j + 1, k) + Ww(i, j + 1, k - 1)) / g.dzf[k];
        const double dtiz = 0.25 * std::fabs(U(i, j, k) + U(i - 1, j, k) + U(i, j, k + 1) + U(i - 1, j, k + 1)) / g.dx +
                            0.25 * std::fabs(Vv(i, j, k) + Vv(i, j - 1, k) + Vv(i, j, k + 1) + Vv(i, j - 1, k + 1)) / g.dy +
                            std::fabs(Ww(i, j, k)) / g.dzc[k + 1];
        dti = std::max(dti, std::max(dtix, std::max(dtiy, dtiz)));
      }
  return dti;
}

}  // namespace

extern "C" {

// Projection u - G L^-1 D u in the box (pressure Neumann at walls, periodic elsewhere).
int oracle_box_project(const int n[3], const int wall[3], const double len_xy[2], const double* dzf, double* u,
                       double* v, double* w, int nthreads) {
  Box g(n, wall, 0.0, len_xy, dzf);
  const size_t N = g.size();
  std::vector<double> d(N), phi(N), gx(N), gy(N), gz(N);
  box_divergence(g, u, v, w, d.data());
  const int bc[3] = {wall[0] ? BC_NN : BC_P, wall[1] ? BC_NN : BC_P, wall[2] ? BC_NN : BC_P};
  int rc = solve_t<double>(n, len_xy, bc, dzf, d.data(), phi.data(), nthreads_or_default(nthreads));
  if (rc) return rc;
  box_gradient(g, phi.data(), gx.data(), gy.data(), gz.data());
  for (size_t c = 0; c < N; ++c) {
    u[c] -= gx[c];
    v[c] -= gy[c];
    w[c] -= gz[c];
  }
  return 0;
}

int oracle_box_divergence(const int n[3], const int wall[3], const double len_xy[2], const double* dzf,
                          const double* u, const double* v, const double* w, double* out) {
  Box g(n, wall, 0.0, len_xy, dzf);
  box_divergence(g, u, v, w, out);
  return 0;
}

// advection (a*) and viscous (l*) operators of the momentum equations in the box
int oracle_box_operators(const int n[3], const int wall[3], double lid, const double len_xy[2], const double* dzf,
                         const double* u, const double* v, const double* w, double* au, double* av, double* aw,
                         double* lu, double* lv, double* lw) {
  Box g(n, wall, lid, len_xy, dzf);
  box_advection(g, u, v, w, au, av, aw);
  box_laplacian(g, u, v, w, lu, lv, lw);
  return 0;
}

// One explicit RK3 fractional step in the box (Eq. up, Eq. poi_ns, correction, p += Phi); dt from
// Eq. dt unless dt_in > 0; forcing != 0 shifts u to the bulk velocity ubulk after each substage.
int oracle_box_rk3_step(const int n[3], const int wall[3], double lid, const double len_xy[2], const double* dzf,
                        double nu, double cfl, double ubulk, int forcing, double dt_in, double* u, double* v,
                        double* w, double* p, double* dt_out, int nthreads) {
  Box g(n, wall, lid, len_xy, dzf);
  const size_t N = g.size();
  double dt = dt_in;
  if (!(dt_in > 0)) {
    double dl = std::min(g.dx, g.dy);
    for (int k = 0; k < g.n[2]; ++k) dl = std::min(dl, g.dzf[k]);
    const double dti = box_max_dti(g, u, v, w);
    dt = 1.65 * dl * dl / nu;
    if (dti > 0) dt = std::min(dt, std::sqrt(3.0) / dti);
    dt *= cfl;
  }
  std::vector<double> au(N), av(N), aw(N), lu(N), lv(N), lw(N), pu(N, 0.0), pv(N, 0.0), pw(N, 0.0);
  std::vector<double> gx(N), gy(N), gz(N), d(N), phi(N);
  const int bc[3] = {wall[0] ? BC_NN : BC_P, wall[1] ? BC_NN : BC_P, wall[2] ? BC_NN : BC_P};
  nthreads = nthreads_or_default(nthreads);
  for (int s = 0; s < 3; ++s) {
    const double a = RK_A[s], b = RK_B[s], gm = a + b;
    box_advection(g, u, v, w, au.data(), av.data(), aw.data());
    box_laplacian(g, u, v, w, lu.data(), lv.data(), lw.data());
    box_gradient(g, p, gx.data(), gy.data(), gz.data());
    for (size_t c = 0; c < N; ++c) {
      const double ru = au[c] + nu * lu[c], rv = av[c] + nu * lv[c], rw = aw[c] + nu * lw[c];
      u[c] += dt * (a * ru + b * pu[c] - gm * gx[c]);
      v[c] += dt * (a * rv + b * pv[c] - gm * gy[c]);
      w[c] += dt * (a * rw + b * pw[c] - gm * gz[c]);
      pu[c] = ru;
      pv[c] = rv;
      pw[c] = rw;
    }
    box_divergence(g, u, v, w, d.data());
    for (size_t c = 0; c < N; ++c) d[c] /= gm * dt;
    const int rc = solve_t<double>(n, len_xy, bc, dzf, d.data(), phi.data(), nthreads);
    if (rc) return rc;
    box_gradient(g, phi.data(), gx.data(), gy.data(), gz.data());
    for (size_t c = 0; c < N; ++c) {
      u[c] -= gm * dt * gx[c];
      v[c] -= gm * dt * gy[c];
      w[c] -= gm * dt * gz[c];
      p[c] += phi[c];
    }
    if (forcing) {
      double sum = 0, vol = 0;
      for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
          for (int i = 0; i < g.n[0]; ++i) {
            sum += g.dzf[k] * u[g.at(i, j, k)];
            vol += g.dzf[k];
          }
      const double shift = ubulk - sum / vol;
      for (size_t c = 0; c < N; ++c) u[c] += shift;
    }
  }
  if (dt_out) *dt_out = dt;
  return 0;
}

}  // extern "C"
