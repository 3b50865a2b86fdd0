// B300 (sm_103a) pressure-Poisson solver by eigenfunction expansion (Eq. poi, Eq. poi_reduced):
// plan construction and the C ABI.  A solve is an x-pass (forward transform along contiguous x
// lines), a y-pass (forward transform along y on tiles of consecutive x-slots), a z-pass (one
// tridiagonal solve per mode), then the inverse y- and x-passes.  Plain mode runs every pass in
// FP64 in place in p; mixed mode runs the passes in FP32 with a double-float residual / iterate and
// FP64 z-solves for the smallest-|mu| modes.  The pass kernels live in kern_*.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "plan.cuh"
#include "wline.cuh"

using namespace cans;

static constexpr int MAXV = 8;  // must match the pass kernels

namespace {
int autotune_plan(cans_plan_s* P);
}

namespace {

int factor_radices(int M, int* radix, int* nst) {
  *nst = 0;
  if (M <= 1) return 0;
  int r = M;
  int n3 = 0, n2 = 0;
  while (r % 3 == 0) { r /= 3; ++n3; }
  while (r % 2 == 0) { r /= 2; ++n2; }
  if (r != 1) return -1;
  for (int i = 0; i < n3; ++i) radix[(*nst)++] = 3;
  while (n2 >= 3) { radix[(*nst)++] = 8; n2 -= 3; }
  if (n2 == 2) radix[(*nst)++] = 4;
  if (n2 == 1) radix[(*nst)++] = 2;
  return (*nst <= 16) ? 0 : -1;
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// eigenvalue of the 1-D second-difference operator (unit spacing) for transform slot s
long double slot_lambda(int bc, int N, int s) {
  const long double pi = 3.141592653589793238462643383279502884L;
  long double th;
  if (bc == BC_P)  // slot 0: k = 0, slot 1: k = N/2, slots 2k, 2k+1: k
    th = pi * (long double)((N > 1 && s == 1) ? N / 2 : s / 2) / N;
  else if (bc == BC_NN)
    th = pi * (long double)s / (2.0L * N);
  else if (bc == BC_DD)
    th = pi * (long double)(s + 1) / (2.0L * N);
  else  // quarter-wave (ND, DN): slot s = mode s
    th = pi * (long double)(2 * s + 1) / (4.0L * N);
  const long double sn = sinl(th);
  return -4.0L * sn * sn;
}

Launch line_launch(int N, int nlines_or_cols, size_t elem2, int prefer_nl) {
  Launch L;
  const int M = std::max(N / 2, 1);
  int nl = prefer_nl;
  while (nl > 1 && (size_t)(nl + 1) * M * elem2 > (size_t)96 * 1024) nl >>= 1;
  while (nl > 1 && nl * M > MAXV * 512) nl >>= 1;
  const int need = 1 << ilog2(std::max(nlines_or_cols, 1));
  while (nl > 1 && nl / 2 >= need) nl >>= 1;
  L.nl = nl;
  L.lognl = ilog2(nl);
  int th = (nl * M + MAXV - 1) / MAXV;
  const int J = MAXV / 2 + 2;
  th = std::max(th, (int)(((M / 2 + 1) * nl + J - 1) / J));
  th = std::max(32, ((th + 31) / 32) * 32);
  L.threads = std::min(th, 512);
  L.smem = (size_t)(nl + 1) * M * elem2;
  return L;
}

template <typename T>
void fill_line_tab(LineTab<T>& t, const DirHost& d, const void* tw, const void* post, const void* mak) {
  t.tw = reinterpret_cast<const typename V2<T>::t*>(tw);
  t.post = reinterpret_cast<const typename V2<T>::t*>(post);
  t.mak = reinterpret_cast<const typename V2<T>::t*>(mak);
  t.n = d.n;
  t.m = d.m;
  t.bc = d.bc;
  t.nst = d.nst;
  for (int i = 0; i < 16; ++i) t.radix[i] = d.radix[i];
}

// one device allocation holding every table; returns byte offsets via a simple bump allocator
struct Bump {
  std::vector<unsigned char> host;
  size_t add(const void* src, size_t bytes) {
    size_t off = (host.size() + 255) & ~size_t(255);
    host.resize(off + bytes);
    std::memcpy(host.data() + off, src, bytes);
    return off;
  }
};

void dir_tables(const DirHost& d, std::vector<double>& tw, std::vector<double>& post, std::vector<double>& mak) {
  const long double pi = 3.141592653589793238462643383279502884L;
  const int M = std::max(d.m, 1), N = d.n;
  tw.assign(2 * M, 0.0);
  post.assign(2 * (M + 1), 0.0);
  mak.assign(2 * (M + 1), 0.0);
  for (int t = 0; t < M; ++t) {
    const long double th = -2.0L * pi * t / M;
    tw[2 * t] = (double)cosl(th);
    tw[2 * t + 1] = (double)sinl(th);
  }
  if (d.bc == BC_ND || d.bc == BC_DN) {  // quarter-wave: post-twiddle exp(-i pi k/N), pre-twiddle exp(-i pi (4m+1)/4N)
    for (int k = 0; k < M; ++k) {
      const long double th = -pi * k / N;
      post[2 * k] = (double)cosl(th);
      post[2 * k + 1] = (double)sinl(th);
      const long double tm = -pi * (4.0L * k + 1.0L) / (4.0L * N);
      mak[2 * k] = (double)cosl(tm);
      mak[2 * k + 1] = (double)sinl(tm);
    }
    return;
  }
  for (int k = 0; k <= M; ++k) {
    const long double th = -2.0L * pi * k / N;
    post[2 * k] = (double)cosl(th);
    post[2 * k + 1] = (double)sinl(th);
    const long double tm = -pi * k / (2.0L * N);
    mak[2 * k] = (double)cosl(tm);
    mak[2 * k + 1] = (double)sinl(tm);
  }
}

std::vector<float> to_float(const std::vector<double>& v) {
  std::vector<float> r(v.size());
  for (size_t i = 0; i < v.size(); ++i) r[i] = (float)v[i];
  return r;
}

void split_df(const std::vector<double>& v, std::vector<float>& hi, std::vector<float>& lo) {
  hi.resize(v.size());
  lo.resize(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    hi[i] = (float)v[i];
    lo[i] = (float)(v[i] - (double)hi[i]);
  }
}


size_t field_points(const cans_plan_s* P) { return (size_t)P->n[0] * P->n[1] * P->n[2]; }

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" {

void cans_opts_default(cans_opts* o) {
  if (!o) return;
  o->prec = CANS_FP64;
  o->max_sweeps = 2;
  o->tol = 1e-12;
  o->fp64_mode_fraction = 0.01;
  o->autotune = 0;
  o->shift = 0.0;
  o->z_grid = 0;
  o->verify = 0;
}

const char* cans_status_string(int s) {
  switch (s) {
    case CANS_OK: return "ok";
    case CANS_ERR_ARG: return "invalid argument";
    case CANS_ERR_UNSUPPORTED: return "unsupported problem for this build";
    case CANS_ERR_CUDA: return "CUDA runtime error";
    case CANS_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case CANS_ERR_INCOMPATIBLE: return "right-hand side incompatible with a singular problem";
    case CANS_ERR_NOT_CONVERGED: return "refinement did not reach the tolerance";
    case CANS_ERR_TIMEOUT: return "bounded device wait timed out";
    default: return "unknown status";
  }
}

int cans_poisson_plan(const int n[3], const double len_xy[2], const int bc[3], const double* dzf,
                      const cans_opts* opts, cans_plan_t* out) {
  if (!n || !len_xy || !bc || !out) return CANS_ERR_ARG;
  *out = nullptr;
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 1) return CANS_ERR_ARG;
    if (bc[d] < 0 || bc[d] > 4) return CANS_ERR_ARG;
  }
  for (int d = 0; d < 2; ++d)
    if (!(len_xy[d] > 0) || !std::isfinite(len_xy[d])) return CANS_ERR_ARG;
  cans_opts o;
  cans_opts_default(&o);
  if (opts) o = *opts;
  if (o.prec != CANS_FP64 && o.prec != CANS_MIXED) return CANS_ERR_ARG;
  if (o.max_sweeps < 0 || o.max_sweeps > 8) return CANS_ERR_ARG;
  if (!(o.fp64_mode_fraction >= 0 && o.fp64_mode_fraction <= 1)) return CANS_ERR_ARG;
  if (!std::isfinite(o.shift) || o.shift > 0) return CANS_ERR_ARG;
  if (o.z_grid != 0 && o.z_grid != 1) return CANS_ERR_ARG;
  if (o.z_grid == 1 && (bc[2] != BC_DD || n[2] < 2)) return CANS_ERR_ARG;
  if (o.verify != 0 && o.verify != 1) return CANS_ERR_ARG;
  const int ncell = n[2];
  std::vector<double> dzcell(ncell);
  for (int k = 0; k < ncell; ++k) {
    dzcell[k] = dzf ? dzf[k] : 1.0 / ncell;
    if (!(dzcell[k] > 0) || !std::isfinite(dzcell[k])) return CANS_ERR_ARG;
  }
  // The solved z grid: widths dz of its control volumes and the distances dzc between consecutive
  // unknowns (dzc[k] between k-1 and k, k = 0..nz; dzc[0] and dzc[nz] reach the mirrored wall
  // ghosts).  Cell centres: the wall ghost mirrors the wall cell, dzc = dzf there.  Interior faces
  // (z_grid 1): unknown k sits on the face between cells k and k+1, its control volume spans the two
  // half cells, neighbouring faces are one cell apart, and a ghost at twice the wall distance with
  // the Dirichlet sign puts w = 0 exactly on the wall face.
  const int nz = ncell - o.z_grid;
  std::vector<double> dz(nz), dzc(nz + 1);
  if (o.z_grid == 0) {
    dz = dzcell;
    for (int k = 1; k < nz; ++k) dzc[k] = 0.5 * (dz[k - 1] + dz[k]);
    dzc[0] = dz[0];
    dzc[nz] = dz[nz - 1];
  } else {
    for (int k = 0; k < nz; ++k) dz[k] = 0.5 * (dzcell[k] + dzcell[k + 1]);
    for (int k = 1; k < nz; ++k) dzc[k] = dzcell[k];
    dzc[0] = 2.0 * dzcell[0];
    dzc[nz] = 2.0 * dzcell[ncell - 1];
  }
  if (bc[2] == BC_P) {
    for (int k = 1; k < nz; ++k)
      if (dz[k] != dz[0]) return CANS_ERR_ARG;
    if (nz > 1 && (nz % 2)) return CANS_ERR_UNSUPPORTED;
    if (nz > 1024) return CANS_ERR_UNSUPPORTED;
  }
  for (int d = 0; d < 2; ++d) {
    if (n[d] > 1 && (n[d] % 2)) return CANS_ERR_UNSUPPORTED;
    if (n[d] > 8192) return CANS_ERR_UNSUPPORTED;
  }
  if (bc[2] != BC_P && nz > 512) return CANS_ERR_UNSUPPORTED;
  if ((size_t)n[0] * n[1] * n[2] >= ((size_t)1 << 40)) return CANS_ERR_UNSUPPORTED;

  cans_plan_s* P = new (std::nothrow) cans_plan_s();
  if (!P) return CANS_ERR_ARG;
  std::memcpy(P->n, n, sizeof(P->n));
  P->n[2] = nz;
  P->nz_cells = ncell;
  std::memcpy(P->len, len_xy, sizeof(P->len));
  std::memcpy(P->bc, bc, sizeof(P->bc));
  P->opts = o;
  P->wblk = 0;  // the blocked work-field layout measured no faster on B300; kept selectable
  cudaGetDevice(&P->device);
  P->sing_bc = (bc[0] == BC_P || bc[0] == BC_NN) && (bc[1] == BC_P || bc[1] == BC_NN) && (bc[2] == BC_P || bc[2] == BC_NN);
  P->shift = o.shift;
  P->singular = P->sing_bc && P->shift == 0.0;

  DirHost* dirs[2] = {&P->dx, &P->dy};
  for (int d = 0; d < 2; ++d) {
    DirHost& D = *dirs[d];
    D.n = n[d];
    D.bc = bc[d];
    D.m = (n[d] >= 2) ? n[d] / 2 : 0;
    if (factor_radices(D.m, D.radix, &D.nst) != 0) {
      delete P;
      return CANS_ERR_UNSUPPORTED;
    }
  }
  if (bc[2] == BC_P) {  // uniform periodic z is diagonalised as well
    P->dz.n = nz;
    P->dz.bc = BC_P;
    P->dz.m = (nz >= 2) ? nz / 2 : 0;
    if (factor_radices(P->dz.m, P->dz.radix, &P->dz.nst) != 0) {
      delete P;
      return CANS_ERR_UNSUPPORTED;
    }
  }
  // eigenvalue terms per slot
  const double hx = len_xy[0] / n[0], hy = len_xy[1] / n[1];
  P->mux_h.resize(n[0]);
  P->muy_h.resize(n[1]);
  for (int s = 0; s < n[0]; ++s) P->mux_h[s] = (double)(slot_lambda(bc[0], n[0], s) / ((long double)hx * hx));
  for (int s = 0; s < n[1]; ++s) P->muy_h[s] = (double)(slot_lambda(bc[1], n[1], s) / ((long double)hy * hy));
  // one cell: the ghosts alone (Dirichlet -c, Neumann c, periodic c itself) give -4, -2 or 0
  auto one_cell = [](int b) { return b == BC_DD ? -4.0 : ((b == BC_ND || b == BC_DN) ? -2.0 : 0.0); };
  if (n[0] == 1) P->mux_h[0] = one_cell(bc[0]) / (hx * hx);
  if (n[1] == 1) P->muy_h[0] = one_cell(bc[1]) / (hy * hy);
  P->idx2 = 1.0 / (hx * hx);
  P->idy2 = 1.0 / (hy * hy);

  // z stencil and tridiagonal rows on the solved grid (dzc with the wall ghosts from above)
  std::vector<double> sa(nz), sc(nz), za(nz), zb(nz), zc(nz);
  for (int k = 0; k < nz; ++k) {
    sa[k] = 1.0 / (dz[k] * dzc[k]);
    sc[k] = 1.0 / (dz[k] * dzc[k + 1]);
    za[k] = sa[k];
    zc[k] = sc[k];
    zb[k] = -(sa[k] + sc[k]);
  }
  // per wall: a Neumann ghost mirrors the wall cell (that flux vanishes), a Dirichlet ghost is its negative
  zb[0] += (bc_lo(bc[2]) == BC_NN) ? sa[0] : -sa[0];
  zb[nz - 1] += (bc_hi(bc[2]) == BC_NN) ? sc[nz - 1] : -sc[nz - 1];
  za[0] = 0;
  zc[nz - 1] = 0;

  // tables -> one device block
  Bump B;
  std::vector<double> tw[2], post[2], mak[2];
  size_t o_tw_d[2], o_post_d[2], o_mak_d[2], o_tw_f[2], o_post_f[2], o_mak_f[2];
  for (int d = 0; d < 2; ++d) {
    dir_tables(*dirs[d], tw[d], post[d], mak[d]);
    o_tw_d[d] = B.add(tw[d].data(), tw[d].size() * 8);
    o_post_d[d] = B.add(post[d].data(), post[d].size() * 8);
    o_mak_d[d] = B.add(mak[d].data(), mak[d].size() * 8);
    auto twf = to_float(tw[d]), postf = to_float(post[d]), makf = to_float(mak[d]);
    o_tw_f[d] = B.add(twf.data(), twf.size() * 4);
    o_post_f[d] = B.add(postf.data(), postf.size() * 4);
    o_mak_f[d] = B.add(makf.data(), makf.size() * 4);
  }
  // stage twiddles of the warp-per-line engine for the float x and y transforms it takes
  size_t o_wst[2] = {0, 0};
  bool has_wst[2] = {false, false};
  for (int d = 0; d < 2; ++d) {
    const int M = dirs[d]->m;
    if (!wl::supported(M)) continue;
    const long double pi = 3.141592653589793238462643383279502884L;
    std::vector<float> wst;
    for (int s = 1; s < wl::nstages(M); ++s) {
      const int R = wl::radix(M, s), Ns = wl::stride(M, s);
      for (int r = 1; r < R; ++r)
        for (int k = 0; k < Ns; ++k) {
          const long double th = -2.0L * pi * k * r / ((long double)R * Ns);
          wst.push_back((float)cosl(th));
          wst.push_back((float)sinl(th));
        }
    }
    o_wst[d] = B.add(wst.data(), wst.size() * 4);
    has_wst[d] = true;
  }
  const size_t o_mux_d = B.add(P->mux_h.data(), n[0] * 8), o_muy_d = B.add(P->muy_h.data(), n[1] * 8);
  auto muxf = to_float(P->mux_h), muyf = to_float(P->muy_h);
  const size_t o_mux_f = B.add(muxf.data(), n[0] * 4), o_muy_f = B.add(muyf.data(), n[1] * 4);
  const size_t o_dzf = B.add(dz.data(), nz * 8);
  std::vector<float> dzff, dzflo;
  split_df(dz, dzff, dzflo);
  std::vector<double> dzfi(nz), dzci(nz);
  for (int k = 0; k < nz; ++k) {
    dzfi[k] = 1.0 / dz[k];
    dzci[k] = 1.0 / dzc[k + 1];
  }
  const size_t o_dzfi = B.add(dzfi.data(), nz * 8), o_dzci = B.add(dzci.data(), nz * 8);
  P->dzf_h = dz;
  const size_t o_dzff = B.add(dzff.data(), nz * 4);
  const size_t o_dzflo = B.add(dzflo.data(), nz * 4);
  const size_t o_sa = B.add(sa.data(), nz * 8), o_sc = B.add(sc.data(), nz * 8);
  std::vector<float> sahi, salo, schi, sclo;
  split_df(sa, sahi, salo);
  split_df(sc, schi, sclo);
  const size_t o_sahi = B.add(sahi.data(), nz * 4), o_salo = B.add(salo.data(), nz * 4);
  const size_t o_schi = B.add(schi.data(), nz * 4), o_sclo = B.add(sclo.data(), nz * 4);
  const size_t o_za = B.add(za.data(), nz * 8), o_zb = B.add(zb.data(), nz * 8), o_zc = B.add(zc.data(), nz * 8);
  auto zaf = to_float(za), zbf = to_float(zb), zcf = to_float(zc);
  const size_t o_zaf = B.add(zaf.data(), nz * 4), o_zbf = B.add(zbf.data(), nz * 4), o_zcf = B.add(zcf.data(), nz * 4);
  size_t o_tz_d = 0, o_post_zd = 0, o_mak_zd = 0, o_tz_f = 0, o_post_zf = 0, o_mak_zf = 0, o_muz_d = 0, o_muz_f = 0;
  if (bc[2] == BC_P) {
    std::vector<double> twz, postz, makz;
    dir_tables(P->dz, twz, postz, makz);
    o_tz_d = B.add(twz.data(), twz.size() * 8);
    o_post_zd = B.add(postz.data(), postz.size() * 8);
    o_mak_zd = B.add(makz.data(), makz.size() * 8);
    auto twzf = to_float(twz), postzf = to_float(postz), makzf = to_float(makz);
    o_tz_f = B.add(twzf.data(), twzf.size() * 4);
    o_post_zf = B.add(postzf.data(), postzf.size() * 4);
    o_mak_zf = B.add(makzf.data(), makzf.size() * 4);
    std::vector<double> muz(nz);
    const double hz = dz[0];
    for (int s = 0; s < nz; ++s) muz[s] = (nz == 1) ? 0.0 : (double)(slot_lambda(BC_P, nz, s) / ((long double)hz * hz));
    auto muzf = to_float(muz);
    o_muz_d = B.add(muz.data(), nz * 8);
    o_muz_f = B.add(muzf.data(), nz * 4);
  }
  size_t o_mask = 0;
  bool has_mask = false;
  if (o.prec == CANS_MIXED) {
    // the ceil(fraction * Nx * Ny) slots with the smallest |mu| (ties by linear index) solve in double
    const size_t ncol = (size_t)n[0] * n[1];
    size_t want = (size_t)std::ceil(o.fp64_mode_fraction * (double)ncol);
    want = std::min(std::max(want, (size_t)1), ncol);
    std::vector<std::pair<double, uint32_t>> keyed(ncol);
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        const size_t c = (size_t)j * n[0] + i;
        keyed[c] = {std::fabs(P->mux_h[i] + P->muy_h[j] + o.shift), (uint32_t)c};
      }
    std::nth_element(keyed.begin(), keyed.begin() + (want - 1), keyed.end());
    std::vector<unsigned char> mask(ncol, 0);
    for (size_t q = 0; q < want; ++q) {
      const uint32_t c = keyed[q].second;
      mask[c] = 1;
      P->mask_i_end = std::max(P->mask_i_end, (int)(c % n[0]) + 1);
      P->mask_j_end = std::max(P->mask_j_end, (int)(c / n[0]) + 1);
    }
    o_mask = B.add(mask.data(), ncol);
    has_mask = true;
  }
  // [0] |f|^2, [1+s] |r_s|^2 (s < max_sweeps), [nacc-7] compatibility sum, [nacc-5] gauge sum,
  // [nacc-4..] reports: slots 1 + max_sweeps .. nacc-8 stay free for every max_sweeps >= 0
  P->nacc = 2 * (o.max_sweeps + 4);
  std::vector<double> zeros(P->nacc, 0.0);
  const size_t o_acc = B.add(zeros.data(), P->nacc * 8);
  const int status0 = CANS_OK;
  const size_t o_status = B.add(&status0, sizeof(int));
  // slots of the reproducible block sums (gauge, bulk velocity): every grid that sums has at most one
  // block per x line, or at most 148 * 16 blocks
  P->dsum_nslots = std::max<size_t>((size_t)n[1] * n[2], (size_t)148 * 16);
  const size_t o_dsum = B.add(std::vector<double>(P->dsum_nslots, 0.0).data(), P->dsum_nslots * sizeof(double));
  const unsigned count0 = 0;
  const size_t o_dcount = B.add(&count0, sizeof(unsigned));
  {
    double w2 = 0;
    for (int k = 0; k < nz; ++k) w2 += dz[k] * dz[k];
    P->compat_scale = std::sqrt((double)n[0] * (double)n[1] * w2);
  }

  if (cudaMalloc(&P->dtab, B.host.size()) != cudaSuccess ||
      cudaMemcpy(P->dtab, B.host.data(), B.host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    if (P->dtab) cudaFree(P->dtab);
    delete P;
    return CANS_ERR_CUDA;
  }
  unsigned char* base = static_cast<unsigned char*>(P->dtab);
  fill_line_tab<double>(P->tx_d, P->dx, base + o_tw_d[0], base + o_post_d[0], base + o_mak_d[0]);
  fill_line_tab<double>(P->ty_d, P->dy, base + o_tw_d[1], base + o_post_d[1], base + o_mak_d[1]);
  fill_line_tab<float>(P->tx_f, P->dx, base + o_tw_f[0], base + o_post_f[0], base + o_mak_f[0]);
  fill_line_tab<float>(P->ty_f, P->dy, base + o_tw_f[1], base + o_post_f[1], base + o_mak_f[1]);
  if (has_wst[0]) P->tx_f.wst = reinterpret_cast<const float2*>(base + o_wst[0]);
  if (has_wst[1]) P->ty_f.wst = reinterpret_cast<const float2*>(base + o_wst[1]);
  P->mux_d = reinterpret_cast<const double*>(base + o_mux_d);
  P->muy_d = reinterpret_cast<const double*>(base + o_muy_d);
  P->mux_f = reinterpret_cast<const float*>(base + o_mux_f);
  P->muy_f = reinterpret_cast<const float*>(base + o_muy_f);
  P->dzf_d = reinterpret_cast<const double*>(base + o_dzf);
  P->dzf_f = reinterpret_cast<const float*>(base + o_dzff);
  P->dzf_flo = reinterpret_cast<const float*>(base + o_dzflo);
  P->dzfi_d = reinterpret_cast<const double*>(base + o_dzfi);
  P->dzci_d = reinterpret_cast<const double*>(base + o_dzci);
  {
    // column mean target: a (0,0) value v contributes v * cx * cy / (Nx Ny) to every cell, with
    // cx = 1 for a periodic or single-cell direction and 1/2 for a Neumann one (DCT-II of a constant)
    const double cx = (bc[0] == BC_NN && n[0] > 1) ? 0.5 : 1.0;
    const double cy = (bc[1] == BC_NN && n[1] > 1) ? 0.5 : 1.0;
    double wsum = 0;
    for (int k = 0; k < nz; ++k) wsum += dz[k];
    P->gauge_scale = -1.0 / (wsum * cx * cy);
  }
  P->sa_d = reinterpret_cast<const double*>(base + o_sa);
  P->sc_d = reinterpret_cast<const double*>(base + o_sc);
  P->sa_hi = reinterpret_cast<const float*>(base + o_sahi);
  P->sa_lo = reinterpret_cast<const float*>(base + o_salo);
  P->sc_hi = reinterpret_cast<const float*>(base + o_schi);
  P->sc_lo = reinterpret_cast<const float*>(base + o_sclo);
  P->zt_d = {reinterpret_cast<const double*>(base + o_za), reinterpret_cast<const double*>(base + o_zb),
             reinterpret_cast<const double*>(base + o_zc)};
  P->zt_f = {reinterpret_cast<const float*>(base + o_zaf), reinterpret_cast<const float*>(base + o_zbf),
             reinterpret_cast<const float*>(base + o_zcf)};
  P->mask_d = has_mask ? base + o_mask : nullptr;
  if (bc[2] == BC_P) {
    fill_line_tab<double>(P->tz_d, P->dz, base + o_tz_d, base + o_post_zd, base + o_mak_zd);
    fill_line_tab<float>(P->tz_f, P->dz, base + o_tz_f, base + o_post_zf, base + o_mak_zf);
    P->muz_d = reinterpret_cast<const double*>(base + o_muz_d);
    P->muz_f = reinterpret_cast<const float*>(base + o_muz_f);
    P->zs_l[0] = line_launch(nz, n[0], sizeof(double2), 8);
    P->zs_l[1] = line_launch(nz, n[0], sizeof(float2), 16);
  }
  P->acc_d = reinterpret_cast<double*>(base + o_acc);
  P->status_d = reinterpret_cast<int*>(base + o_status);
  P->dsum_slots = reinterpret_cast<double*>(base + o_dsum);
  P->dsum_count = reinterpret_cast<unsigned*>(base + o_dcount);

  // launch shapes
  const int nlines = n[1] * nz;
  P->x_l[0] = line_launch(n[0], nlines, sizeof(double2), 16);
  P->x_l[1] = line_launch(n[0], nlines, sizeof(float2), 32);
  P->y_l[0] = line_launch(n[1], n[0], sizeof(double2), 8);
  P->y_l[1] = line_launch(n[1], n[0], sizeof(float2), 16);
  // rows per lane: the power of two >= Nz/32 (rows past Nz are identity rows)
  P->z_mmax = 1;
  while (32 * P->z_mmax < nz) P->z_mmax <<= 1;
  P->z_m = P->z_mmax;
  for (int s = 0; s < 2; ++s) {
    int ti = (s == 0) ? 16 : 32;
    const size_t es = (s == 0) ? 8 : 4;
    while (ti > 1 && (size_t)ti * nz * es > (size_t)96 * 1024) ti >>= 1;
    while (ti > 1 && ti / 2 >= n[0]) ti >>= 1;
    P->z_ti[s] = ti;
    P->z_smem[s] = (size_t)ti * nz * es;
  }
  // CANS_RES_PTS=1/2/4 sets the residual stencil's points per thread, CANS_Z_P2=0 keeps the float z pass of
  // full columns on the staged kernel, CANS_Z_FUSE64=0 / 2 keeps the marked columns of short ones in the
  // separate double kernel / fuses them at every field size, CANS_RES_SPLIT=0 / 2 keeps the sweep residual of CTA-engine x lines
  // fused into the x pass / splits it at every size (switches for comparisons and tests).  CANS_Z_TMA=0 keeps the float z pass on the register-staged kernel, =2 makes a shape the
  // TMA kernel cannot take fail instead of falling back (switches for comparisons and tests; the
  // autotuner, when on, chooses between the two kernels by timing)
  if (const char* ev = std::getenv("CANS_RES_PTS")) P->res_pts = (ev[0] == '1') ? 1 : (ev[0] == '2' ? 2 : 4);
  if (const char* ev = std::getenv("CANS_Z_P2")) P->z_p2 = (ev[0] == '0') ? 0 : 1;
  if (const char* ev = std::getenv("CANS_Z_FUSE64")) P->z_fuse64 = (ev[0] == '0') ? 0 : (ev[0] == '2' ? 2 : 1);
  if (const char* ev = std::getenv("CANS_RES_SPLIT")) P->res_split = (ev[0] == '0') ? 0 : (ev[0] == '2' ? 2 : 1);
  if (const char* ev = std::getenv("CANS_Z_TMA")) P->z_tma = (ev[0] == '0') ? 0 : (ev[0] == '2' ? 2 : 1);
  if (const char* ev = std::getenv("CANS_Z_TMA_CTAS"))
    P->z_tma_ctas = (ev[0] >= '1' && ev[0] <= '4') ? ev[0] - '0' : P->z_tma_ctas;
  if (o.autotune) {
    const int rc = autotune_plan(P);
    if (rc != CANS_OK) {
      cudaFree(P->dtab);
      delete P;
      return rc;
    }
  }
  *out = P;
  return CANS_OK;
}

// Mixed-path workspace: the float work field W (blocked layout, x padded to a multiple of 32 slots),
// then the double-float iterate Phi, Plo (natural layout).
static size_t work_field_bytes(const cans_plan_s* P) {
  const size_t nxp = P->wblk ? (size_t)((P->n[0] + 31) / 32) * 32 : (size_t)P->n[0];
  return align256(nxp * P->n[1] * P->n[2] * sizeof(float));
}

int cans_poisson_workspace_size(cans_plan_t P, size_t* bytes) {
  if (!P || !bytes) return CANS_ERR_ARG;
  const size_t N = field_points(P);
  *bytes = (P->opts.prec == CANS_MIXED) ? work_field_bytes(P) + 2 * align256(N * sizeof(float)) : 0;
  return CANS_OK;
}

int cans_poisson_adjoint_workspace_size(cans_plan_t P, size_t* bytes) {
  if (!P || !bytes) return CANS_ERR_ARG;
  size_t b = 0;
  cans_poisson_workspace_size(P, &b);
  *bytes = align256(b) + align256(field_points(P) * sizeof(double));
  return CANS_OK;
}

int cans_poisson_solve_adjoint(cans_plan_t P, const double* g, double* q, void* workspace, void* cuda_stream) {
  if (!P || !g || !q) return CANS_ERR_ARG;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) return CANS_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  size_t b = 0;
  cans_poisson_workspace_size(P, &b);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  double* t = reinterpret_cast<double*>(ws + align256(b));
  // S^T = D S D^-1, D = diag(dzf_k): the solve is self-adjoint in the dzf-weighted inner product
  if (launch_scale_z(P, g, t, P->dzfi_d, st) != cudaSuccess) return CANS_ERR_CUDA;
  // a scaled g is generically incompatible in the singular case: project it exactly in FP64 (the
  // solve projects too, but the mixed path would do it in float); S Pi = S, the result is unchanged
  if (P->singular && launch_remove_weighted_mean(P, t, P->acc_d + P->nacc - 2, st) != cudaSuccess) return CANS_ERR_CUDA;
  const int rc = cans_poisson_solve(P, t, q, b ? workspace : nullptr, cuda_stream, nullptr);
  if (rc != CANS_OK) return rc;
  if (launch_scale_z(P, q, q, P->dzf_d, st) != cudaSuccess) return CANS_ERR_CUDA;
  return CANS_OK;
}

int cans_plan_destroy(cans_plan_t P) {
  if (!P) return CANS_ERR_ARG;
  for (cudaEvent_t e : P->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : P->host_ev)
    if (e) cudaEventDestroy(e);
  if (P->dtab) cudaFree(P->dtab);
  delete P;
  return CANS_OK;
}

int cans_plan_profile(cans_plan_t P, int enable) {
  if (!P) return CANS_ERR_ARG;
  P->profiling = enable != 0;
  if (enable) {
    P->ev_used = 0;
    P->ev_kind.clear();
  }
  return CANS_OK;
}

int cans_plan_profile_read(cans_plan_t P, int pass, double* total_ms, int* launches) {
  if (!P || pass < 0 || pass >= CANS_PASS_COUNT || !total_ms || !launches) return CANS_ERR_ARG;
  double tot = 0;
  int cnt = 0;
  for (int r = 0; r < P->ev_used; ++r) {
    if (P->ev_kind[r] != pass) continue;
    if (cudaEventSynchronize(P->ev_pool[2 * r + 1]) != cudaSuccess) return CANS_ERR_CUDA;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, P->ev_pool[2 * r], P->ev_pool[2 * r + 1]) != cudaSuccess) return CANS_ERR_CUDA;
    tot += ms;
    ++cnt;
  }
  *total_ms = tot;
  *launches = cnt;
  return CANS_OK;
}

int cans_plan_eigenvalues(cans_plan_t P, double* mux, double* muy) {
  if (!P) return CANS_ERR_ARG;
  if (mux) std::memcpy(mux, P->mux_h.data(), sizeof(double) * P->n[0]);
  if (muy) std::memcpy(muy, P->muy_h.data(), sizeof(double) * P->n[1]);
  return CANS_OK;
}

}  // extern "C"

namespace {

}  // namespace

Launch cans::line_launch_shape(int N, int count, size_t elem2, int prefer_nl) {
  return line_launch(N, count, elem2, prefer_nl);
}

cudaError_t cans::set_smem(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::mutex lock;
  static std::vector<std::pair<std::pair<const void*, int>, size_t>> done;  // (kernel, device) -> bytes
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> guard(lock);
  for (auto& d : done)
    if (d.first.first == fn && d.first.second == dev && d.second >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  for (auto& d : done)
    if (d.first.first == fn && d.first.second == dev) {
      d.second = bytes;
      return cudaSuccess;
    }
  done.push_back({{fn, dev}, bytes});
  return cudaSuccess;
}

// Each pass is an NVTX range (seen by Nsight tools attached to the process; a no-op otherwise) and,
// while cans_plan_profile is on, a pair of CUDA events on the pass's stream.
namespace {
const char* const kPassName[CANS_PASS_COUNT] = {
    "x_forward",        "y_forward",        "z_solve",          "y_inverse",  "x_inverse",
    "x_forward_residual", "x_inverse_update", "residual_stencil", "z_solve_double_columns",
    "momentum",         "divergence",       "correction",       "chkdt",      "forcing"};
}  // namespace

cans::PassTimer::PassTimer(cans_plan_s* P_, int kind, cudaStream_t st_) : P(P_), st(st_) {
  nvtxRangePushA(kPassName[kind]);
  if (!P->profiling) return;
  if ((size_t)(2 * P->ev_used + 2) > P->ev_pool.size()) {
    for (int q = 0; q < 64; ++q) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      P->ev_pool.push_back(e);
    }
  }
  rec = P->ev_used++;
  P->ev_kind.push_back(kind);
  cudaEventRecord(P->ev_pool[2 * rec], st);
}

cans::PassTimer::~PassTimer() {
  if (rec >= 0) cudaEventRecord(P->ev_pool[2 * rec + 1], st);
  nvtxRangePop();
}

namespace {

#define CK(...)                                  \
  do {                                           \
    cudaError_t e_ = (__VA_ARGS__);              \
    if (e_ != cudaSuccess) return CANS_ERR_CUDA; \
  } while (0)

}  // namespace

// ---- autotuner ---------------------------------------------------------------------------------
// With opts.autotune = 1 the plan times candidate tile shapes for each pass on scratch fields (CUDA
// events, best of 3 launches after a warm-up) and keeps the fastest: lines per CTA of the x and y
// passes (and of the spectral z pass), x-slots per CTA of the tridiagonal z pass.  Results are cached
// per (device, shape, boundary conditions, precision) for the life of the process and, when the
// environment variable CANS_AUTOTUNE_CACHE names a file, read from and appended to that file.
namespace {

std::mutex g_tune_lock;
std::vector<std::pair<std::string, std::vector<int>>> g_tune_cache;

std::string tune_key(const cans_plan_s* P) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev);
  auto I = [](int v) { return std::to_string(v); };
  std::string k = std::string(prop.name) + "|" + I(P->n[0]) + "," + I(P->n[1]) + "," + I(P->n[2]) + "|" + I(P->bc[0]) +
                  "," + I(P->bc[1]) + "," + I(P->bc[2]) + "|" + I(P->opts.prec);
  for (char& ch : k)
    if (ch == ' ') ch = '_';
  return k;
}

bool tune_lookup(const std::string& key, std::vector<int>& v) {
  std::lock_guard<std::mutex> g(g_tune_lock);
  for (auto& e : g_tune_cache)
    if (e.first == key) {
      v = e.second;
      return true;
    }
  const char* path = std::getenv("CANS_AUTOTUNE_CACHE");
  if (!path) return false;
  FILE* fh = std::fopen(path, "r");
  if (!fh) return false;
  char line[512];
  bool found = false;
  while (std::fgets(line, sizeof(line), fh)) {
    char k[400];
    int a, b, cc, d, t = 0;
    const int got = std::sscanf(line, "%399s %d %d %d %d %d", k, &a, &b, &cc, &d, &t);
    if (got >= 5 && key == k) {
      v = {a, b, cc, d, got == 6 ? t : 0};
      found = true;
    }
  }
  std::fclose(fh);
  if (found) g_tune_cache.push_back({key, v});
  return found;
}

void tune_store(const std::string& key, const std::vector<int>& v) {
  std::lock_guard<std::mutex> g(g_tune_lock);
  g_tune_cache.push_back({key, v});
  const char* path = std::getenv("CANS_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* fh = std::fopen(path, "a");
  if (!fh) return;
  std::fprintf(fh, "%s %d %d %d %d %d\n", key.c_str(), v[0], v[1], v[2], v[3], v[4]);
  std::fclose(fh);
}

template <typename F>
float time_best(F&& launch) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  launch();
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(a, 0);
    cudaError_t e = launch();
    cudaEventRecord(b, 0);
    cudaEventSynchronize(b);
    float ms = 1e30f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

int autotune_plan(cans_plan_s* P) {
  const int s = (P->opts.prec == CANS_FP64) ? 0 : 1;
  const size_t es = s ? sizeof(float2) : sizeof(double2);
  const std::string key = tune_key(P);
  std::vector<int> v;
  auto apply = [&](const std::vector<int>& c) {
    const int nlines = P->n[1] * P->n[2];
    P->x_l[s] = line_launch(P->n[0], nlines, es, c[0]);
    P->y_l[s] = line_launch(P->n[1], P->n[0], es, c[1]);
    if (P->bc[2] == BC_P) {
      P->zs_l[s] = line_launch(P->n[2], P->n[0], es, c[2]);
    } else {
      P->z_ti[s] = c[3];
      P->z_smem[s] = (size_t)c[3] * P->n[2] * (s ? 4 : 8);
      if (s) {
        P->z_tma = c[4] ? 1 : 0;
        if (c[4]) P->z_tma_ctas = c[4];
      }
    }
  };
  if (tune_lookup(key, v)) {
    apply(v);
    return CANS_OK;
  }
  const size_t N = (size_t)P->n[0] * P->n[1] * P->n[2];
  double* f = nullptr;
  void* w = nullptr;
  if (cudaMalloc(&f, N * sizeof(double)) != cudaSuccess) return CANS_ERR_CUDA;
  const size_t wbytes = s ? work_field_bytes(P) : N * 8;
  if (cudaMalloc(&w, wbytes) != cudaSuccess) {
    cudaFree(f);
    return CANS_ERR_CUDA;
  }
  cudaMemset(f, 0, N * sizeof(double));
  cudaMemset(w, 0, wbytes);
  std::vector<int> best = {P->x_l[s].nl, P->y_l[s].nl, P->zs_l[s].nl, P->z_ti[s], 0};
  const int cand_nl[4] = {4, 8, 16, 32};
  const int cand_ti[3] = {s ? 8 : 4, s ? 16 : 8, s ? 32 : 16};
  const int nlines = P->n[1] * P->n[2];
  float bx = 1e30f, by = 1e30f, bz = 1e30f;
  for (int c : cand_nl) {
    P->x_l[s] = line_launch(P->n[0], nlines, es, c);
    const float t = s ? time_best([&] { return launch_xfwd<float, 0>(P, f, nullptr, nullptr, (float*)w, nullptr, 0); })
                      : time_best([&] { return launch_xfwd<double, 0>(P, f, nullptr, nullptr, (double*)w, nullptr, 0); });
    if (t < bx) { bx = t; best[0] = c; }
    P->y_l[s] = line_launch(P->n[1], P->n[0], es, c);
    const float ty = s ? time_best([&] { return launch_y<float, 1>(P, (float*)w, 0); })
                       : time_best([&] { return launch_y<double, 1>(P, (double*)w, 0); });
    if (ty < by) { by = ty; best[1] = c; }
    if (P->bc[2] == BC_P) {
      P->zs_l[s] = line_launch(P->n[2], P->n[0], es, c);
      const float tz = s ? time_best([&] { return launch_z<float>(P, (float*)w, nullptr, 0); })
                         : time_best([&] { return launch_z<double>(P, (double*)w, nullptr, 0); });
      if (tz < bz) { bz = tz; best[2] = c; }
    }
  }
  if (P->bc[2] != BC_P) {
    P->z_tma = 0;
    for (int ti : cand_ti) {
      if ((size_t)ti * P->n[2] * (s ? 4 : 8) > (size_t)96 * 1024) continue;
      P->z_ti[s] = ti;
      P->z_smem[s] = (size_t)ti * P->n[2] * (s ? 4 : 8);
      const float tz = s ? time_best([&] { return launch_z<float>(P, (float*)w, nullptr, 0); })
                         : time_best([&] { return launch_z<double>(P, (double*)w, nullptr, 0); });
      if (tz < bz) { bz = tz; best[3] = ti; }
    }
    if (s && ztma_feasible(P, w)) {  // the TMA-fed float kernel (tile width fixed), 2 or 3 CTAs per SM
      P->z_tma = 1;
      for (int ctas : {4, 1, 2, 3}) {
        P->z_tma_ctas = ctas;
        const float tz = time_best([&] { return launch_z<float>(P, (float*)w, nullptr, 0); });
        if (tz < bz) { bz = tz; best[4] = ctas; }
      }
    }
  }
  cudaFree(f);
  cudaFree(w);
  apply(best);
  tune_store(key, best);
  return (cudaGetLastError() == cudaSuccess) ? CANS_OK : CANS_ERR_CUDA;
}

}  // namespace

extern "C" {

// The solve, with its right-hand side either read from f or (div != NULL) formed as the divergence of a
// channel's face velocities inside the first x pass; f is then the optional by-product array.
static int solve_impl(cans_plan_t P, const double* f, const DivArgs* div, double* p, void* workspace,
                      void* cuda_stream, double* info) {
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t N = field_points(P);
  const int sweeps = P->opts.max_sweeps;
  const double inv_scale = 1.0 / ((double)P->n[0] * P->n[1]);
#define TIMED(kind, ...)                    \
  do {                                      \
    PassTimer tm_(P, kind, st);             \
    CK(__VA_ARGS__);                        \
  } while (0)
  // the z pass of the mixed path: the float columns, then the double ones (lowest |mu|, singular)
  auto z_pass = [&](float* W, const double* gz, double* cp) -> int {
    TIMED(CANS_PASS_Z, launch_z<float>(P, W, gz, st, 0, cp));
    TIMED(CANS_PASS_ZD, launch_z<float>(P, W, gz, st, 1, cp));
    return CANS_OK;
  };
  // the singular column's weighted sum before its projection (compatibility check of the status word)
  double* compat = P->singular ? P->acc_d + P->nacc - 7 : nullptr;
  if (P->opts.prec == CANS_FP64) {
    CK(cudaMemsetAsync(P->acc_d, 0, P->nacc * sizeof(double), st));
    if (div)
      TIMED(CANS_PASS_XF, launch_xfwd_div<double>(P, *div, p, P->acc_d, st));
    else
      TIMED(CANS_PASS_XF, launch_xfwd<double, 0>(P, f, nullptr, nullptr, p, P->acc_d, st));
    TIMED(CANS_PASS_YF, launch_y<double, 1>(P, p, st));
    TIMED(CANS_PASS_Z, launch_z<double>(P, p, nullptr, st, -1, compat));
    TIMED(CANS_PASS_YI, launch_y<double, -1>(P, p, st));
    TIMED(CANS_PASS_XI, launch_xinv<double, 0>(P, p, p, nullptr, nullptr, inv_scale, nullptr, st));
  } else {
    if (f == p || (f == nullptr && sweeps > 0)) return CANS_ERR_ARG;  // the residual re-reads f
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) return CANS_ERR_WORKSPACE;
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    float* W = reinterpret_cast<float*>(ws);
    float* Phi = reinterpret_cast<float*>(ws + work_field_bytes(P));
    float* Plo = reinterpret_cast<float*>(ws + work_field_bytes(P) + align256(N * 4));
    CK(cudaMemsetAsync(P->acc_d, 0, P->nacc * sizeof(double), st));
    if (div)
      TIMED(CANS_PASS_XF, launch_xfwd_div<float>(P, *div, W, P->acc_d, st));
    else
      TIMED(CANS_PASS_XF, launch_xfwd<float, 0>(P, f, nullptr, nullptr, W, P->acc_d, st));
    TIMED(CANS_PASS_YF, launch_y<float, 1>(P, W, st));
    if (const int rz = z_pass(W, nullptr, compat)) return rz;
    TIMED(CANS_PASS_YI, launch_y<float, -1>(P, W, st));
    if (sweeps == 0) {
      TIMED(CANS_PASS_XI, launch_xinv<float, 0>(P, W, p, nullptr, nullptr, inv_scale, nullptr, st));
    } else {
      double* gauge = P->singular ? P->acc_d + P->nacc - 5 : nullptr;
      TIMED(CANS_PASS_XI, launch_xinv<float, 1>(P, W, nullptr, Phi, Plo, inv_scale, gauge, st));
      for (int s = 0; s < sweeps; ++s) {
        // residual r = f - L_h(Phi + Plo) transformed along x: a streaming stencil + in-place transform
        // where the x lines fit the warp-per-line kernels, else one CTA-wide kernel with both fused
        if (xres_warp_ok(P, W)) {
          TIMED(CANS_PASS_RS, launch_residual(P, f, Phi, Plo, s > 0, W, P->acc_d + 1 + s, st));
          TIMED(CANS_PASS_XR, launch_xfwd32_warp(P, W, st));
        } else if ((P->res_split == 2 || (P->res_split == 1 && N >= ((size_t)1 << 24))) && xres_cta_ok(P, W)) {
          // large fields: the stencil + a float x pass (measured 2.04 vs 2.23 ms at 192x512x512);
          // small ones keep the fused pass, one launch fewer on their latency-bound chain
          TIMED(CANS_PASS_RS, launch_residual(P, f, Phi, Plo, s > 0, W, P->acc_d + 1 + s, st));
          TIMED(CANS_PASS_XR, launch_xfwd32_cta(P, W, st));
        } else if (s == 0) {
          TIMED(CANS_PASS_XR, launch_xfwd<float, 2>(P, f, Phi, Plo, W, P->acc_d + 1 + s, st));
        } else {
          TIMED(CANS_PASS_XR, launch_xfwd<float, 1>(P, f, Phi, Plo, W, P->acc_d + 1 + s, st));
        }
        TIMED(CANS_PASS_YF, launch_y<float, 1>(P, W, st));
        if (const int rz = z_pass(W, s == 0 ? gauge : nullptr, nullptr)) return rz;
        TIMED(CANS_PASS_YI, launch_y<float, -1>(P, W, st));
        const bool last = (s + 1 == sweeps);
        if (s == 0 && !last)
          TIMED(CANS_PASS_XU, launch_xinv<float, 4>(P, W, nullptr, Phi, Plo, inv_scale, nullptr, st));
        else if (s == 0)
          TIMED(CANS_PASS_XU, launch_xinv<float, 5>(P, W, p, Phi, Plo, inv_scale, nullptr, st));
        else if (!last)
          TIMED(CANS_PASS_XU, launch_xinv<float, 2>(P, W, nullptr, Phi, Plo, inv_scale, nullptr, st));
        else
          TIMED(CANS_PASS_XU, launch_xinv<float, 3>(P, W, p, Phi, Plo, inv_scale, nullptr, st));
      }
    }
  }
  // the final residual (opts.verify, or a caller that asks for the norms; not for an in-place FP64
  // solve, whose f is gone), then the status word's checks
  double* acc2 = P->acc_d + P->nacc - 4;
  const bool verify = (info != nullptr || P->opts.verify) && f != nullptr && f != p;
  if (verify) CK(launch_residual_norms(P, f, p, acc2, st));
  CK(launch_solve_status(P, compat != nullptr, verify, st));
  if (info) {
    if (P->singular && verify) CK(launch_weighted_sum(P, f, acc2 + 2, st));
    std::vector<double> h(P->nacc);
    int word = CANS_OK;
    const int zero = CANS_OK;
    CK(cudaMemcpyAsync(h.data(), P->acc_d, P->nacc * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&word, P->status_d, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(P->status_d, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    const double rr = h[P->nacc - 4], ff = h[P->nacc - 3];
    const double fn = std::sqrt(ff);
    if (P->opts.prec == CANS_MIXED) {
      for (int s = 0; s < sweeps; ++s) info[s] = std::sqrt(h[1 + s]) / fn;
      info[sweeps] = std::sqrt(rr) / fn;
      info[sweeps + 1] = std::sqrt(rr) / fn;
    } else {
      info[0] = std::sqrt(rr) / fn;
      for (int s = 1; s < sweeps + 2; ++s) info[s] = info[0];
    }
    if (!verify) {  // in place: f is gone, no residual to report (the device checks still ran)
      for (int s = 0; s < sweeps + 2; ++s) info[s] = std::nan("");
      return word;
    }
    if (P->singular && std::fabs(h[P->nacc - 2]) > 1e-10 * h[P->nacc - 1]) return CANS_ERR_INCOMPATIBLE;
    if (P->opts.prec == CANS_MIXED && info[sweeps] > P->opts.tol) return CANS_ERR_NOT_CONVERGED;
    if (word != CANS_OK) return word;
  }
  return CANS_OK;
}

int cans_poisson_solve(cans_plan_t P, const double* f, double* p, void* workspace, void* cuda_stream, double* info) {
  if (!P || !f || !p) return CANS_ERR_ARG;
  return solve_impl(P, f, nullptr, p, workspace, cuda_stream, info);
}

int cans_poisson_solve_host(cans_plan_t P, const double* f_host, double* p_host, double* f_dev, double* p_dev,
                            void* workspace, void* copy_in_stream, void* compute_stream, void* copy_out_stream) {
  if (!P || !f_host || !p_host || !f_dev || !p_dev || f_dev == p_dev) return CANS_ERR_ARG;
  if (P->opts.prec == CANS_MIXED && (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)))
    return CANS_ERR_WORKSPACE;  // refused before the upload is enqueued
  cudaStream_t sin = static_cast<cudaStream_t>(copy_in_stream), sc = static_cast<cudaStream_t>(compute_stream),
               sout = static_cast<cudaStream_t>(copy_out_stream);
  for (cudaEvent_t& e : P->host_ev)
    if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return CANS_ERR_CUDA;
  const size_t bytes = field_points(P) * sizeof(double);
  // upload on copy_in, solve on compute after it, download on copy_out after the solve: each stream
  // waits only for what it consumes, so consecutive calls with other device buffers overlap
  if (cudaMemcpyAsync(f_dev, f_host, bytes, cudaMemcpyHostToDevice, sin) != cudaSuccess ||
      cudaEventRecord(P->host_ev[0], sin) != cudaSuccess || cudaStreamWaitEvent(sc, P->host_ev[0], 0) != cudaSuccess)
    return CANS_ERR_CUDA;
  const int rc = solve_impl(P, f_dev, nullptr, p_dev, workspace, compute_stream, nullptr);
  if (rc != CANS_OK) return rc;
  if (cudaEventRecord(P->host_ev[1], sc) != cudaSuccess || cudaStreamWaitEvent(sout, P->host_ev[1], 0) != cudaSuccess ||
      cudaMemcpyAsync(p_host, p_dev, bytes, cudaMemcpyDeviceToHost, sout) != cudaSuccess)
    return CANS_ERR_CUDA;
  return CANS_OK;
}

int cans_poisson_solve_divergence(cans_plan_t P, const double* u, const double* v, const double* w, double scale,
                                  const double* dt_dev, double gamma, double* f, double* p, void* workspace,
                                  void* cuda_stream, double* info) {
  if (!P || !u || !v || !w || !p) return CANS_ERR_ARG;
  if (P->bc[0] != BC_P || P->bc[1] != BC_P || P->bc[2] != BC_NN || P->opts.z_grid != 0) return CANS_ERR_UNSUPPORTED;
  if (dt_dev != nullptr && !(gamma != 0.0)) return CANS_ERR_ARG;
  if (f != nullptr && (f == p || f == u || f == v || f == w)) return CANS_ERR_ARG;
  if (p == u || p == v || p == w) return CANS_ERR_ARG;
  const DivArgs d = div_args(P, u, v, w, f, scale, dt_dev, gamma);
  return solve_impl(P, f, &d, p, workspace, cuda_stream, info);
}

int cans_plan_status(cans_plan_t P, int* status) {
  if (!P || !status) return CANS_ERR_ARG;
  *status = CANS_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CANS_ERR_CUDA;
  if (dev != P->device && cudaSetDevice(P->device) != cudaSuccess) return CANS_ERR_CUDA;
  int word = CANS_OK;
  const int zero = CANS_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&word, P->status_d, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(P->status_d, &zero, sizeof(int), cudaMemcpyHostToDevice);
  if (dev != P->device) cudaSetDevice(dev);
  if (e != cudaSuccess) return CANS_ERR_CUDA;
  *status = word;
  return CANS_OK;
}

int cans_helmholtz_solve(cans_plan_t P, const double* f, double* p, double shift, void* workspace,
                         void* cuda_stream, double* info) {
  if (!P) return CANS_ERR_ARG;
  if (!std::isfinite(shift) || shift > 0) return CANS_ERR_ARG;
  const double shift0 = P->shift;
  P->shift = shift;  // read by the launches of this call (kernel arguments), restored after
  P->singular = P->sing_bc && shift == 0.0;
  const int rc = cans_poisson_solve(P, f, p, workspace, cuda_stream, info);
  P->shift = shift0;
  P->singular = P->sing_bc && shift0 == 0.0;
  return rc;
}

int cans_transform_xy(cans_plan_t P, double* field, int dir, void* cuda_stream) {
  if (!P || !field || (dir != 1 && dir != -1)) return CANS_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (dir > 0) {
    CK(launch_xfwd<double, 0>(P, field, nullptr, nullptr, field, nullptr, st));
    CK((launch_y<double, 1>(P, field, st)));
  } else {
    CK((launch_y<double, -1>(P, field, st)));
    // inverse x without the 1/(Nx Ny) normalisation
    CK((launch_xinv<double, 0>(P, field, field, nullptr, nullptr, 1.0, nullptr, st)));
  }
  return CANS_OK;
}

int cans_transform_xy_f32(cans_plan_t P, double* field, float* work, int dir, void* cuda_stream) {
  if (!P || !field || !work || (dir != 1 && dir != -1)) return CANS_ERR_ARG;
  if (P->opts.prec != CANS_MIXED || P->wblk) return CANS_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (dir > 0) {
    CK((launch_xfwd<float, 0>(P, field, nullptr, nullptr, work, nullptr, st)));
    CK((launch_y<float, 1>(P, work, st)));
  } else {
    CK((launch_y<float, -1>(P, work, st)));
    CK((launch_xinv<float, 0>(P, work, field, nullptr, nullptr, 1.0, nullptr, st)));
  }
  return CANS_OK;
}

int cans_zsolve(cans_plan_t P, double* field, void* cuda_stream) {
  if (!P || !field) return CANS_ERR_ARG;
  CK(launch_z<double>(P, field, nullptr, static_cast<cudaStream_t>(cuda_stream)));
  return CANS_OK;
}

}  // extern "C"
