// nbgb_api.cu -- the C ABI of libnbgb (declared in include/nbgb.h): the
// handle, argument checks, the per-shot host set-up (rotated axes per phi
// step and mosaic domain, source tables, panel offsets) and the launches.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/nbgb.h"
#include "nbgb_internal.cuh"

using nbgb::DevPanel;
using nbgb::SpotArgs;

namespace {

// NB_OPT_FAIL_ALLOCS: how many of the library's next device allocations
// fail as if the device were out of memory (a test hook, process-wide)
std::atomic<long long> g_fail_allocs{0};

bool inject_alloc_failure() {
  long long left = g_fail_allocs.load();
  while (left > 0)
    if (g_fail_allocs.compare_exchange_weak(left, left - 1)) return true;
  return false;
}

struct DevBuf {
  void *p = nullptr;
  size_t n = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    if (bytes == 0) return cudaSuccess;
    if (inject_alloc_failure()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) n = bytes;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

struct nb_sim {
  int device = 0;
  int precision = NB_MIXED;
  cudaStream_t stream = nullptr;
  std::string err;
  // state flags
  bool have_crystal = false, have_F = false, have_beam = false,
       have_det = false;
  // crystal (host copies)
  double axes[9] = {0};
  std::vector<double> umats;
  int n_mosaic = 0, n_phi = 1;
  double phi0 = 0, phistep = 0, spindle[3] = {0, 1, 0};
  double N[3] = {1, 1, 1};
  int shape = NB_SHAPE_SINC;
  double scale = 1.0;
  int hmin[3] = {0, 0, 0}, hn[3] = {0, 0, 0};
  int interp = NB_INTERP_NEAREST;
  double defF = 0.0;
  // beam
  std::vector<double> dirs, lam, w;
  int n_src = 0;
  double fluence = 0, kahn = 0, evec[3] = {1, 0, 0};
  // detector
  std::vector<nb_panel> panels;
  std::vector<long long> pix0;
  long long npix = 0;
  int n_tiles = 0;
  int os = 1, T = 1;
  double thick = 0, atten = 0;
  // device
  DevBuf d_panels, d_ax64, d_axh, d_axl, d_src64, d_src32, d_divh, d_divl,
      d_F, d_image, d_list, d_tmp, d_stats, d_work, d_srcq, d_check;
  float sinc_qG = 0.f;  // grid of G for the sinc fast path (0: off)
  float sinc_dq[2] = {0.f, 0.f};  // range of the sources' delta on its grid
  int variant = NB_VARIANT_AUTO;
  int sm_count = 0;
  long long last_pixel_steps = 0, last_pixels = 0;
  bool last_warp = false;  // the last launch ran the warp-per-pixel kernel
  bool count_work = false;  // NB_OPT_COUNT_WORK
  bool last_counted = false;  // the last launch counted its work
  // parametrised crystal (for gradients): U, cell, rotation angles
  bool have_params = false;
  double pU[9] = {0}, pcell[3] = {0}, prot[3] = {0};
  double daxes[6][9];  // d(lab axes)/d(tx, ty, tz, a, b, c)
  DevBuf d_dax, d_part, d_grad, d_F4, d_C4, d_F64t;
  bool F4_valid = false, C4_valid = false, F64_valid = false;
  int has_div = 0;
  double u0 = 0;
  bool tables_dirty = true;
  // amorphous background: knots, scattering factors, molecules in the beam
  bool have_bg = false;
  std::vector<double> bg_stol, bg_F;
  double bg_nmol = 0;
  DevBuf d_bg64, d_bg32, d_bgrng;
};

static int fail(nb_sim *s, int code, const std::string &msg) {
  if (s) s->err = msg;
  return code;
}

static int cuda_fail(nb_sim *s, cudaError_t e, const char *what) {
  return fail(s, NB_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

static bool finite3(const double *v) {
  return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

static double norm3(const double *v) {
  return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
}

// ------------------------------------------------------------ host set-up

// Rotation by `ang` radians about the unit axis k, as a 3x3 matrix:
// R = I + sin(ang) K + (1 - cos(ang)) K^2 with K the cross-product matrix.
static void axis_rotation(const double *k, double ang, double *R) {
  double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double v = 0;
      for (int l = 0; l < 3; ++l) v += K[3 * i + l] * K[3 * l + j];
      K2[3 * i + j] = v;
    }
  double sn = std::sin(ang), cs = 1.0 - std::cos(ang);
  for (int i = 0; i < 9; ++i)
    R[i] = (i % 4 == 0 ? 1.0 : 0.0) + sn * K[i] + cs * K2[i];
}

namespace nbgb {
// rows (a, b, c) of U_m R_phi(j) lab for all (j, m): ax[pm][9]
void rotated_axes_table(const double *lab, const double *umats, int n_mosaic,
                        int n_phi, double phi0_deg, double phistep_deg,
                        const double *spindle, std::vector<double> &ax) {
  int PM = n_phi * n_mosaic;
  ax.assign((size_t)PM * 9, 0.0);
  double k[3] = {0, 1, 0};
  double nk = norm3(spindle);
  if (nk > 0)
    for (int i = 0; i < 3; ++i) k[i] = spindle[i] / nk;
  for (int j = 0; j < n_phi; ++j) {
    double R[9];
    axis_rotation(k, (phi0_deg + j * phistep_deg) * (M_PI / 180.0), R);
    for (int m = 0; m < n_mosaic; ++m) {
      const double *U = umats + 9 * m;
      double UR[9];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
          UR[3 * r + c] = U[3 * r] * R[c] + U[3 * r + 1] * R[3 + c] +
                          U[3 * r + 2] * R[6 + c];
      double *out = ax.data() + ((size_t)j * n_mosaic + m) * 9;
      for (int v = 0; v < 3; ++v)
        for (int r = 0; r < 3; ++r)
          out[3 * v + r] = UR[3 * r] * lab[3 * v] +
                           UR[3 * r + 1] * lab[3 * v + 1] +
                           UR[3 * r + 2] * lab[3 * v + 2];
    }
  }
}
}  // namespace nbgb

static void build_axes_of(const nb_sim *s, const double *lab,
                          std::vector<double> &ax) {
  nbgb::rotated_axes_table(lab, s->umats.data(), s->n_mosaic, s->n_phi,
                           s->phi0, s->phistep, s->spindle, ax);
}

static void build_axes(const nb_sim *s, std::vector<double> &ax) {
  build_axes_of(s, s->axes, ax);
}

// 3x3 row-major product C = A B
static void mat3_mul(const double *A, const double *B, double *C) {
  double T[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      T[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] +
                     A[3 * i + 2] * B[6 + j];
  std::memcpy(C, T, sizeof T);
}

// elementary rotation about axis `ax` (0 x, 1 y, 2 z) by t, or its
// derivative with respect to t
static void elem_rot(int ax, double t, bool deriv, double *M) {
  double c = std::cos(t), s = std::sin(t);
  double dc = -s, ds = c;
  if (deriv) {
    c = dc;
    s = ds;
  }
  double one = deriv ? 0.0 : 1.0;
  double R[9] = {0};
  int i = (ax + 1) % 3, j = (ax + 2) % 3;
  R[3 * ax + ax] = one;
  R[3 * i + i] = c;
  R[3 * i + j] = -s;
  R[3 * j + i] = s;
  R[3 * j + j] = c;
  std::memcpy(M, R, sizeof R);
}

// lab axes (rows a, b, c) = rows of Rx(tx) Ry(ty) Rz(tz) U diag(cell), i.e.
// axis v = cell_v times column v of R U; and their derivatives
static void param_axes(const double *U, const double *cell, const double *rot,
                       double *axes, double dax[6][9]) {
  double Rx[9], Ry[9], Rz[9], D[3][9];
  elem_rot(0, rot[0], false, Rx);
  elem_rot(1, rot[1], false, Ry);
  elem_rot(2, rot[2], false, Rz);
  double RU[9], dRU[3][9], T[9];
  mat3_mul(Ry, Rz, T);
  mat3_mul(Rx, T, RU);
  mat3_mul(RU, U, RU);
  for (int r = 0; r < 3; ++r) {
    double Rs[3][9];
    std::memcpy(Rs[0], Rx, sizeof Rx);
    std::memcpy(Rs[1], Ry, sizeof Ry);
    std::memcpy(Rs[2], Rz, sizeof Rz);
    elem_rot(r, rot[r], true, D[r]);
    std::memcpy(Rs[r], D[r], sizeof D[r]);
    mat3_mul(Rs[1], Rs[2], T);
    mat3_mul(Rs[0], T, dRU[r]);
    mat3_mul(dRU[r], U, dRU[r]);
  }
  for (int v = 0; v < 3; ++v)
    for (int c = 0; c < 3; ++c) axes[3 * v + c] = cell[v] * RU[3 * c + v];
  for (int r = 0; r < 6; ++r)
    for (int i = 0; i < 9; ++i) dax[r][i] = 0.0;
  for (int r = 0; r < 3; ++r)
    for (int v = 0; v < 3; ++v)
      for (int c = 0; c < 3; ++c)
        dax[r][3 * v + c] = cell[v] * dRU[r][3 * c + v];
  for (int v = 0; v < 3; ++v)
    for (int c = 0; c < 3; ++c) dax[3 + v][3 * v + c] = RU[3 * c + v];
}

// transverse polarization basis of source direction dir: E' = unit part of
// e normal to dir, B' = dir x E'
static void pol_basis(const double *dir, const double *e, double *ep,
                      double *bp) {
  double de = dir[0] * e[0] + dir[1] * e[1] + dir[2] * e[2];
  for (int i = 0; i < 3; ++i) ep[i] = e[i] - de * dir[i];
  double n = norm3(ep);
  for (int i = 0; i < 3; ++i) ep[i] /= n;
  bp[0] = dir[1] * ep[2] - dir[2] * ep[1];
  bp[1] = dir[2] * ep[0] - dir[0] * ep[2];
  bp[2] = dir[0] * ep[1] - dir[1] * ep[0];
}

static void split_ff(double v, float &hi, float &lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

namespace nbgb {
// Reorders the sources by ascending 1/lambda (stable).  The sum over
// sources does not depend on their order; sorted wavenumbers let the
// warp-per-pixel kernel turn a wavenumber interval into a source range.
void sort_sources(std::vector<double> &dirs, std::vector<double> &lam,
                  std::vector<double> &w) {
  size_t S = lam.size();
  std::vector<size_t> idx(S);
  for (size_t i = 0; i < S; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
    return 1.0 / lam[a] < 1.0 / lam[b];
  });
  std::vector<double> d2(3 * S), l2(S), w2(S);
  for (size_t i = 0; i < S; ++i) {
    for (int c = 0; c < 3; ++c) d2[3 * i + c] = dirs[3 * idx[i] + c];
    l2[i] = lam[idx[i]];
    w2[i] = w[idx[i]];
  }
  dirs.swap(d2);
  lam.swap(l2);
  w.swap(w2);
}

// u0 = centre of the 1/lambda range of the sources
double source_u0(const double *lam, int S) {
  double umin = 1e300, umax = -1e300;
  for (int k = 0; k < S; ++k) {
    double u = 1.0 / lam[k];
    umin = std::fmin(umin, u);
    umax = std::fmax(umax, u);
  }
  return 0.5 * (umin + umax);
}

// FP32 tables of one shot: double-float axes [PM][9] and the source rows
// [S][SRC32_STRIDE] (delta = 1/lambda - u0 split, w, dir, E', B')
void shot_tables_f32(const std::vector<double> &ax, const double *lam,
                     const double *w, const double *dirs, int S,
                     const double *evec, double u0, bool plain_f32,
                     std::vector<float> &axh, std::vector<float> &axl,
                     std::vector<float> &src32) {
  axh.resize(ax.size());
  axl.resize(ax.size());
  for (size_t i = 0; i < ax.size(); ++i) split_ff(ax[i], axh[i], axl[i]);
  src32.assign((size_t)S * SRC32_STRIDE, 0.f);
  for (int k = 0; k < S; ++k) {
    const double *dir = dirs + 3 * k;
    double u = 1.0 / lam[k], ep[3], bp[3];
    pol_basis(dir, evec, ep, bp);
    float *q = src32.data() + (size_t)k * SRC32_STRIDE;
    if (plain_f32) {
      q[SRC32_DH] = 0.f;
      q[SRC32_DL] = (float)u;  // plain FP32 arm reads u_k here
    } else {
      split_ff(u - u0, q[SRC32_DH], q[SRC32_DL]);
    }
    q[SRC32_W] = (float)w[k];
    for (int c = 0; c < 3; ++c) {
      q[SRC32_DIR + c] = (float)dir[c];
      q[SRC32_E + c] = (float)ep[c];
      q[SRC32_B + c] = (float)bp[c];
    }
  }
}
}  // namespace nbgb

// Uploads the crystal x beam tables (they depend on both).
static int upload_tables(nb_sim *s) {
  if (!s->tables_dirty) return NB_OK;
  int PM = s->n_phi * s->n_mosaic, S = s->n_src;
  std::vector<double> ax;
  build_axes(s, ax);
  s->u0 = nbgb::source_u0(s->lam.data(), S);
  std::vector<float> axh, axl, src32;
  nbgb::shot_tables_f32(ax, s->lam.data(), s->w.data(), s->dirs.data(), S,
                        s->evec, s->u0, s->precision == NB_F32, axh, axl,
                        src32);
  std::vector<double> src64((size_t)S * nbgb::SRC64_STRIDE);
  s->has_div = 0;
  for (int k = 0; k < S; ++k) {
    const double *dir = s->dirs.data() + 3 * k;
    for (int c = 0; c < 3; ++c)
      if (dir[c] != s->dirs[c]) s->has_div = 1;
  }
  for (int k = 0; k < S; ++k) {
    const double *dir = s->dirs.data() + 3 * k;
    double u = 1.0 / s->lam[k], ep[3], bp[3];
    pol_basis(dir, s->evec, ep, bp);
    double *r = src64.data() + (size_t)k * nbgb::SRC64_STRIDE;
    r[nbgb::SRC64_LAM] = s->lam[k];
    r[nbgb::SRC64_W] = s->w[k];
    (void)u;
    for (int c = 0; c < 3; ++c) {
      r[nbgb::SRC64_DIR + c] = dir[c];
      r[nbgb::SRC64_E + c] = ep[c];
      r[nbgb::SRC64_B + c] = bp[c];
    }
  }
  // sinc fast path (NB_MIXED, one direction): delta_k = u_k - u0 on the
  // grid qD = 2^(e - 12), |delta| <= 2^e, so that delta / qD has at most
  // 12 bits; the kernel rounds G to qG = 2^-21 / qD, so that the product
  // of the two rounded values is exact in FP32 and lies on the 2^-21 grid
  // of r (see mixed_pixel.cuh)
  std::vector<float> srcq;
  s->sinc_qG = 0.f;
  if (s->precision == NB_MIXED && !s->has_div) {
    double m = 0.0;
    for (int k = 0; k < S; ++k)
      m = std::max(m, std::fabs(1.0 / s->lam[k] - s->u0));
    const int e = m > 0.0 ? (int)std::ceil(std::log2(m)) : -20;
    const double qD = std::ldexp(1.0, e - 12);
    // two float4 per pair of sources 2j, 2j + 1: (delta_q, delta_q,
    // rest, rest) and (w, w, delta, delta); an odd count ends with a copy
    // of the last source of weight 0
    const int P = (S + 1) / 2;
    srcq.assign((size_t)8 * P, 0.f);
    for (int k = 0; k < 2 * P; ++k) {
      const int kk = std::min(k, S - 1), j = k / 2, q = k % 2;
      const double d = 1.0 / s->lam[kk] - s->u0;
      const double dq = std::nearbyint(d / qD) * qD;
      float *r = srcq.data() + (size_t)8 * j;
      r[q] = (float)dq;  // exact: at most 13 bits on a power-of-2 grid
      r[2 + q] = (float)(d - dq);
      r[4 + q] = k < S ? src32[(size_t)k * nbgb::SRC32_STRIDE + nbgb::SRC32_W]
                       : 0.f;
      r[6 + q] = (float)d;
      s->sinc_dq[0] = k ? std::min(s->sinc_dq[0], r[q]) : r[q];
      s->sinc_dq[1] = k ? std::max(s->sinc_dq[1], r[q]) : r[q];
    }
    s->sinc_qG = (float)std::ldexp(1.0, -21 - (e - 12));
  }
  // divergence term E[pm][k][x] = A_pm,x . (i_k - i_0) u_k
  std::vector<float> divh, divl;
  if (s->has_div) {
    divh.resize((size_t)PM * S * 3);
    divl.resize(divh.size());
    for (int pm = 0; pm < PM; ++pm)
      for (int k = 0; k < S; ++k) {
        double di[3], u = 1.0 / s->lam[k];
        for (int c = 0; c < 3; ++c) di[c] = s->dirs[3 * k + c] - s->dirs[c];
        for (int x = 0; x < 3; ++x) {
          const double *A = ax.data() + (size_t)pm * 9 + 3 * x;
          double E = (A[0] * di[0] + A[1] * di[1] + A[2] * di[2]) * u;
          size_t e = ((size_t)pm * S + k) * 3 + x;
          split_ff(E, divh[e], divl[e]);
        }
      }
  }
  cudaError_t e;
  if ((e = s->d_ax64.ensure(ax.size() * 8)) != cudaSuccess ||
      (e = s->d_axh.ensure(axh.size() * 4)) != cudaSuccess ||
      (e = s->d_axl.ensure(axl.size() * 4)) != cudaSuccess ||
      (e = s->d_src64.ensure(src64.size() * 8)) != cudaSuccess ||
      (e = s->d_src32.ensure(src32.size() * 4)) != cudaSuccess)
    return fail(s, NB_ENOMEM, std::string("device tables: ") +
                                  cudaGetErrorString(e));
  cudaMemcpyAsync(s->d_ax64.p, ax.data(), ax.size() * 8,
                  cudaMemcpyHostToDevice, s->stream);
  cudaMemcpyAsync(s->d_axh.p, axh.data(), axh.size() * 4,
                  cudaMemcpyHostToDevice, s->stream);
  cudaMemcpyAsync(s->d_axl.p, axl.data(), axl.size() * 4,
                  cudaMemcpyHostToDevice, s->stream);
  cudaMemcpyAsync(s->d_src64.p, src64.data(), src64.size() * 8,
                  cudaMemcpyHostToDevice, s->stream);
  cudaMemcpyAsync(s->d_src32.p, src32.data(), src32.size() * 4,
                  cudaMemcpyHostToDevice, s->stream);
  if (!srcq.empty()) {
    if ((e = s->d_srcq.ensure(srcq.size() * 4)) != cudaSuccess)
      return fail(s, NB_ENOMEM, "source grid table");
    cudaMemcpyAsync(s->d_srcq.p, srcq.data(), srcq.size() * 4,
                    cudaMemcpyHostToDevice, s->stream);
  }
  if (s->has_div) {
    if ((e = s->d_divh.ensure(divh.size() * 4)) != cudaSuccess ||
        (e = s->d_divl.ensure(divl.size() * 4)) != cudaSuccess)
      return fail(s, NB_ENOMEM, "divergence table");
    cudaMemcpyAsync(s->d_divh.p, divh.data(), divh.size() * 4,
                    cudaMemcpyHostToDevice, s->stream);
    cudaMemcpyAsync(s->d_divl.p, divl.data(), divl.size() * 4,
                    cudaMemcpyHostToDevice, s->stream);
  }
  if (s->have_params) {
    // derivative of every rotated axis: the same rotations applied to the
    // derivative of the lab axes (the maps are linear): [PM][6][9] floats
    std::vector<float> dax((size_t)PM * 54);
    for (int r = 0; r < 6; ++r) {
      std::vector<double> t;
      build_axes_of(s, s->daxes[r], t);
      for (int pm = 0; pm < PM; ++pm)
        for (int i = 0; i < 9; ++i)
          dax[(size_t)pm * 54 + r * 9 + i] = (float)t[(size_t)pm * 9 + i];
    }
    if ((e = s->d_dax.ensure(dax.size() * 4)) != cudaSuccess)
      return fail(s, NB_ENOMEM, "derivative table");
    cudaMemcpyAsync(s->d_dax.p, dax.data(), dax.size() * 4,
                    cudaMemcpyHostToDevice, s->stream);
  }
  // pageable copies are staged before return; check the queue is healthy
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(s, e, "table upload");
  s->tables_dirty = false;
  return NB_OK;
}

static void fill_args(const nb_sim *s, SpotArgs &a) {
  std::memset(&a, 0, sizeof a);
  a.panels = (const DevPanel *)s->d_panels.p;
  a.n_panels = (int)s->panels.size();
  a.n_tiles = s->n_tiles;
  a.npix = s->npix;
  a.os = s->os;
  a.T = s->T;
  a.dt = s->thick > 0 ? s->thick / s->T : 0.0;
  a.thickness = s->thick;
  a.atten = s->atten;
  a.PM = s->n_phi * s->n_mosaic;
  a.ax64 = (const double *)s->d_ax64.p;
  a.axh = (const float *)s->d_axh.p;
  a.axl = (const float *)s->d_axl.p;
  for (int i = 0; i < 3; ++i) {
    a.N64[i] = s->N[i];
    a.N[i] = (float)s->N[i];
    a.hmin[i] = s->hmin[i];
    a.hn[i] = s->hn[i];
    a.i0[i] = s->dirs[i];
  }
  double nn = s->N[0] * s->N[1] * s->N[2];
  a.N6 = (float)(nn * nn);
  a.shape = s->shape;
  a.interp = s->interp;
  a.F = (const float *)s->d_F.p;
  a.F4 = s->F4_valid ? (const float4 *)s->d_F4.p : nullptr;
  a.C4 = s->C4_valid ? (const float4 *)s->d_C4.p : nullptr;
  a.F64t = s->F64_valid ? (const double *)s->d_F64t.p : nullptr;
  a.defF = (float)s->defF;
  a.defF64 = s->defF;
  a.S = s->n_src;
  a.src64 = (const double *)s->d_src64.p;
  a.src32 = (const float *)s->d_src32.p;
  a.u0 = s->u0;
  split_ff(s->u0, a.u0h, a.u0l);
  pol_basis(s->dirs.data(), s->evec, a.e0, a.b0);
  a.kahn = (float)s->kahn;
  a.kahn64 = s->kahn;
  a.has_div = s->has_div;
  a.divh = (const float *)s->d_divh.p;
  a.divl = (const float *)s->d_divl.p;
  a.srcq = s->sinc_qG > 0.f ? (const float *)s->d_srcq.p : nullptr;
  a.sinc_qG = a.srcq ? s->sinc_qG : 0.f;
  a.sinc_dq[0] = s->sinc_dq[0];
  a.sinc_dq[1] = s->sinc_dq[1];
  a.prefactor = nbgb::kElectronRadius * nbgb::kElectronRadius * s->fluence *
                s->scale / ((double)s->os * s->os * s->n_mosaic * s->n_phi);
  a.image = (double *)s->d_image.p;
  a.check = (unsigned long long *)s->d_check.p;  // NB_CHECK builds only
  nbgb::args_ff(a);
}

// NB_CHECK builds: waits for the handle's work and reports a failed bounds
// check of its kernels (the site and index the first one recorded)
static int read_check(nb_sim *s) {
#if NB_CHECK
  if (!s->d_check.p) return NB_OK;
  unsigned long long w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, s->d_check.p, sizeof w,
                                  cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "bounds-check read");
  if (w) {
    char msg[128];
    std::snprintf(msg, sizeof msg, "bounds check failed: site %d index %lld",
                  (int)((w >> 56) & 0x7f),
                  (long long)(w & ((1ull << 56) - 1)));
    cudaMemsetAsync(s->d_check.p, 0, sizeof w, s->stream);
    return fail(s, NB_ECUDA, msg);
  }
#else
  (void)s;
#endif
  return NB_OK;
}

// ------------------------------------------------------------------- ABI

extern "C" {

const char *nb_version(void) {
  return NB_CHECK ? "nbgb 0.1 (sm_103a) +check" : "nbgb 0.1 (sm_103a)";
}

const char *nb_last_error(const nb_sim *sim) {
  if (!sim) return "null handle";
  return sim->err.c_str();
}

int nb_sim_create(nb_sim **out, int device, int precision,
                  void *cuda_stream) {
  if (!out) return NB_EINVAL;
  *out = nullptr;
  if (precision < NB_F64 || precision > NB_F32) return NB_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 ||
      device >= ndev) {
    cudaGetLastError();
    return NB_ECUDA;
  }
  nb_sim *s = new (std::nothrow) nb_sim();
  if (!s) return NB_ENOMEM;
  s->device = device;
  s->precision = precision;
  if (cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount,
                             device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return NB_ECUDA;
  }
  s->stream = (cudaStream_t)cuda_stream;
#if NB_CHECK
  {
    // the word a failed bounds check writes
    DeviceGuard g(device);
    if (s->d_check.ensure(sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(s->d_check.p, 0, sizeof(unsigned long long)) !=
            cudaSuccess) {
      cudaGetLastError();
      s->d_check.release();
      delete s;
      return NB_ENOMEM;
    }
  }
#endif
  *out = s;
  return NB_OK;
}

int nb_free(nb_sim *sim) {
  if (!sim) return NB_OK;
  {
    DeviceGuard g(sim->device);
    cudaStreamSynchronize(sim->stream);
    DevBuf *bufs[] = {&sim->d_panels, &sim->d_ax64, &sim->d_axh,
                      &sim->d_axl,    &sim->d_src64, &sim->d_src32,
                      &sim->d_divh,   &sim->d_divl,  &sim->d_F,
                      &sim->d_image,  &sim->d_list,  &sim->d_tmp,
                      &sim->d_stats,  &sim->d_work,  &sim->d_srcq,  &sim->d_check,  &sim->d_dax,
                      &sim->d_part,   &sim->d_grad,  &sim->d_F4,
                      &sim->d_C4,     &sim->d_F64t,  &sim->d_bg64,
                      &sim->d_bg32,   &sim->d_bgrng};
    for (DevBuf *b : bufs) b->release();
  }
  delete sim;
  return NB_OK;
}

int nb_set_crystal(nb_sim *s, const double axes[9], const double *umats,
                   int n_mosaic, int n_phi, double phi0_deg,
                   double phistep_deg, const double spindle[3], double Na,
                   double Nb, double Nc, int shape, const float *F,
                   const int hkl_min[3], const int hkl_n[3], int interp,
                   double default_F) {
  nbgb::NvtxRange nvtx_("nb_set_crystal");
  if (!s) return NB_EINVAL;
  if (!axes || !umats) return fail(s, NB_EINVAL, "axes/umats NULL");
  if (n_mosaic < 1 || n_phi < 1 || (long long)n_mosaic * n_phi > nbgb::kMaxPM)
    return fail(s, NB_EINVAL, "need 1 <= n_mosaic*n_phi <= 2048");
  if (shape != NB_SHAPE_SINC && shape != NB_SHAPE_GAUSS)
    return fail(s, NB_EINVAL, "bad shape");
  double N[3] = {Na, Nb, Nc};
  for (int i = 0; i < 3; ++i) {
    if (!(N[i] > 0) || !std::isfinite(N[i]))
      return fail(s, NB_EINVAL, "N must be positive");
    if (shape == NB_SHAPE_SINC && N[i] != std::floor(N[i]))
      return fail(s, NB_EINVAL, "sinc shape needs integral N");
  }
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(axes[i])) return fail(s, NB_EINVAL, "axes not finite");
  double sp[3] = {0, 1, 0};
  if (spindle) std::memcpy(sp, spindle, sizeof sp);
  if (n_phi > 1 && !(norm3(sp) > 0))
    return fail(s, NB_EINVAL, "zero spindle with n_phi > 1");
  if (F) {
    if (!hkl_min || !hkl_n) return fail(s, NB_EINVAL, "hkl_min/hkl_n NULL");
    for (int i = 0; i < 3; ++i)
      if (hkl_n[i] < 1) return fail(s, NB_EINVAL, "empty structure-factor table");
    if (interp != NB_INTERP_NEAREST && interp != NB_INTERP_TRICUBIC)
      return fail(s, NB_EINVAL, "bad interp");
  } else if (!s->have_F) {
    return fail(s, NB_EINVAL, "no structure-factor table yet");
  }
  DeviceGuard g(s->device);
  std::memcpy(s->axes, axes, sizeof s->axes);
  s->umats.assign(umats, umats + 9 * (size_t)n_mosaic);
  s->n_mosaic = n_mosaic;
  s->n_phi = n_phi;
  s->phi0 = phi0_deg;
  s->phistep = phistep_deg;
  std::memcpy(s->spindle, sp, sizeof sp);
  std::memcpy(s->N, N, sizeof N);
  s->shape = shape;
  if (F) {
    size_t nF = (size_t)hkl_n[0] * hkl_n[1] * hkl_n[2];
    cudaError_t e = s->d_F.ensure(nF * sizeof(float));
    if (e != cudaSuccess) return fail(s, NB_ENOMEM, "F table");
    e = cudaMemcpyAsync(s->d_F.p, F, nF * sizeof(float),
                        cudaMemcpyHostToDevice, s->stream);
    // the caller's array may be pinned: finish the copy before returning
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "F upload");
    for (int i = 0; i < 3; ++i) {
      s->hmin[i] = hkl_min[i];
      s->hn[i] = hkl_n[i];
    }
    s->interp = interp;
    s->defF = default_F;
    s->have_F = true;
    s->F4_valid = false;
    s->C4_valid = false;
    s->F64_valid = false;
  } else {
    if (interp == NB_INTERP_NEAREST || interp == NB_INTERP_TRICUBIC)
      s->interp = interp;
    if (std::isfinite(default_F)) s->defF = default_F;
  }
  s->have_crystal = true;
  s->have_params = false;
  s->tables_dirty = true;
  return NB_OK;
}

int nb_set_fcell_device(nb_sim *s, const float *F, size_t n_elems) {
  nbgb::NvtxRange nvtx_("nb_set_fcell_device");
  if (!s) return NB_EINVAL;
  if (!F) return fail(s, NB_EINVAL, "F NULL");
  if (!s->have_F) return fail(s, NB_ESTATE, "no structure-factor table yet");
  const size_t nF = (size_t)s->hn[0] * s->hn[1] * s->hn[2];
  if (n_elems != nF)
    return fail(s, NB_EINVAL, "n_elems differs from the table's size");
  DeviceGuard g(s->device);
  cudaError_t e = cudaMemcpyAsync(s->d_F.p, F, nF * sizeof(float),
                                  cudaMemcpyDeviceToDevice, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "F copy");
  // the derived tables are rebuilt from the new values at the next launch
  s->F4_valid = false;
  s->C4_valid = false;
  s->F64_valid = false;
  return NB_OK;
}

int nb_set_crystal_params(nb_sim *s, const double U[9], const double cell[3],
                          const double rot[3], const double ncells[3],
                          double scale) {
  nbgb::NvtxRange nvtx_("nb_set_crystal_params");
  if (!s) return NB_EINVAL;
  if (!U || !cell || !rot || !ncells)
    return fail(s, NB_EINVAL, "NULL parameter array");
  if (!s->have_crystal)
    return fail(s, NB_ESTATE, "nb_set_crystal must come first");
  for (int i = 0; i < 3; ++i) {
    if (!(cell[i] > 0) || !std::isfinite(cell[i]) || !std::isfinite(rot[i]))
      return fail(s, NB_EINVAL, "cell / rotation");
    if (!(ncells[i] > 0) || !std::isfinite(ncells[i]) ||
        (s->shape == NB_SHAPE_SINC && ncells[i] != std::floor(ncells[i])))
      return fail(s, NB_EINVAL, "N");
  }
  if (!std::isfinite(scale)) return fail(s, NB_EINVAL, "scale");
  std::memcpy(s->pU, U, sizeof s->pU);
  std::memcpy(s->pcell, cell, sizeof s->pcell);
  std::memcpy(s->prot, rot, sizeof s->prot);
  param_axes(U, cell, rot, s->axes, s->daxes);
  std::memcpy(s->N, ncells, sizeof s->N);
  s->scale = scale;
  s->have_params = true;
  s->tables_dirty = true;
  return NB_OK;
}

int nb_set_scale(nb_sim *s, double scale) {
  if (!s) return NB_EINVAL;
  if (!std::isfinite(scale)) return fail(s, NB_EINVAL, "scale not finite");
  s->scale = scale;
  return NB_OK;
}

int nb_set_beam(nb_sim *s, const double *dirs, const double *lambda_A,
                const double *weights, int n_src, double fluence,
                double kahn_K, const double e_vec[3]) {
  nbgb::NvtxRange nvtx_("nb_set_beam");
  if (!s) return NB_EINVAL;
  if (n_src < 1 || n_src > nbgb::kMaxSrc)
    return fail(s, NB_EINVAL, "need 1 <= n_src <= 1024");
  if (!dirs || !lambda_A || !weights)
    return fail(s, NB_EINVAL, "beam arrays NULL");
  if (!(kahn_K >= 0 && kahn_K <= 1))
    return fail(s, NB_EINVAL, "kahn_K outside [0, 1]");
  if (!std::isfinite(fluence)) return fail(s, NB_EINVAL, "fluence");
  double e[3] = {1, 0, 0};
  if (e_vec) std::memcpy(e, e_vec, sizeof e);
  for (int k = 0; k < n_src; ++k) {
    const double *d = dirs + 3 * k;
    if (!finite3(d) || std::fabs(norm3(d) - 1.0) > 1e-9)
      return fail(s, NB_EINVAL, "source direction not unit");
    if (!(lambda_A[k] > 0) || !std::isfinite(lambda_A[k]))
      return fail(s, NB_EINVAL, "wavelength must be positive");
    if (!std::isfinite(weights[k])) return fail(s, NB_EINVAL, "weight");
    double de = d[0] * e[0] + d[1] * e[1] + d[2] * e[2];
    double t[3] = {e[0] - de * d[0], e[1] - de * d[1], e[2] - de * d[2]};
    if (!(norm3(t) > 1e-6 * norm3(e)))
      return fail(s, NB_EINVAL, "e_vec parallel to a source direction");
  }
  s->dirs.assign(dirs, dirs + 3 * (size_t)n_src);
  s->lam.assign(lambda_A, lambda_A + n_src);
  s->w.assign(weights, weights + n_src);
  nbgb::sort_sources(s->dirs, s->lam, s->w);
  s->n_src = n_src;
  s->fluence = fluence;
  s->kahn = kahn_K;
  std::memcpy(s->evec, e, sizeof e);
  s->have_beam = true;
  s->tables_dirty = true;
  return NB_OK;
}

long long nb_num_pixels(const nb_sim *s) { return s ? s->npix : 0; }

int nb_set_detector(nb_sim *s, int n_panels, const nb_panel *panels,
                    int oversample, int n_layers, double thickness_m,
                    double atten_m) {
  nbgb::NvtxRange nvtx_("nb_set_detector");
  if (!s) return NB_EINVAL;
  if (n_panels < 1 || !panels) return fail(s, NB_EINVAL, "no panels");
  if (oversample < 1 || oversample > 64 || n_layers < 1 || n_layers > 64)
    return fail(s, NB_EINVAL, "oversample / n_layers out of range");
  if (!(thickness_m >= 0) || !std::isfinite(thickness_m))
    return fail(s, NB_EINVAL, "thickness");
  if (thickness_m == 0 && n_layers != 1)
    return fail(s, NB_EINVAL, "layers need a sensor thickness");
  if (thickness_m > 0 && !(atten_m > 0))
    return fail(s, NB_EINVAL, "attenuation length must be positive");
  std::vector<DevPanel> dp(n_panels);
  std::vector<long long> pix0(n_panels);
  long long npix = 0;
  int tiles = 0;
  for (int q = 0; q < n_panels; ++q) {
    const nb_panel &p = panels[q];
    if (p.nfast < 1 || p.nslow < 1 || !(p.pixel_m > 0))
      return fail(s, NB_EINVAL, "panel size");
    if (!finite3(p.origin) || !finite3(p.fdir) || !finite3(p.sdir) ||
        !finite3(p.ndir))
      return fail(s, NB_EINVAL, "panel vectors not finite");
    DevPanel &d = dp[q];
    std::memset(&d, 0, sizeof d);
    for (int c = 0; c < 3; ++c) {
      d.origin[c] = p.origin[c];
      d.fdir[c] = p.fdir[c];
      d.sdir[c] = p.sdir[c];
      d.ndir[c] = p.ndir[c];
    }
    d.px = p.pixel_m;
    d.nfast = p.nfast;
    d.nslow = p.nslow;
    d.pix0 = npix;
    d.tile0 = tiles;
    d.tiles_f = (p.nfast + nbgb::kTileF - 1) / nbgb::kTileF;
    d.tiles = d.tiles_f * ((p.nslow + nbgb::kTileS - 1) / nbgb::kTileS);
    nbgb::panel_ff(d);
    pix0[q] = npix;
    npix += (long long)p.nfast * p.nslow;
    if ((long long)tiles + d.tiles > 2000000000LL)
      return fail(s, NB_EINVAL, "detector too large");
    tiles += d.tiles;
  }
  DeviceGuard g(s->device);
  cudaError_t e = s->d_panels.ensure(dp.size() * sizeof(DevPanel));
  if (e != cudaSuccess) return fail(s, NB_ENOMEM, "panel table");
  e = cudaMemcpyAsync(s->d_panels.p, dp.data(), dp.size() * sizeof(DevPanel),
                      cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "panel upload");
  e = s->d_image.ensure((size_t)npix * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(s, NB_ENOMEM, "image");
  }
  e = cudaMemsetAsync(s->d_image.p, 0, (size_t)npix * sizeof(double),
                      s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "image clear");
  s->panels.assign(panels, panels + n_panels);
  s->pix0 = pix0;
  s->npix = npix;
  s->n_tiles = tiles;
  s->os = oversample;
  s->T = n_layers;
  s->thick = thickness_m;
  s->atten = atten_m;
  s->have_det = true;
  return NB_OK;
}

// 16-byte rows of the F table for tricubic lookups in the FP32 forms
// (4x the table's memory; skipped if that allocation fails)
static void ensure_sliding_table(nb_sim *s) {
  if (s->F4_valid || s->interp != NB_INTERP_TRICUBIC ||
      s->precision == NB_F64)
    return;
  size_t n = (size_t)s->hn[0] * s->hn[1] * s->hn[2];
  if (s->d_F4.ensure(n * sizeof(float4)) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (nbgb::build_sliding_table((const float *)s->d_F.p, s->hn,
                                (float4 *)s->d_F4.p, s->stream) == cudaSuccess)
    s->F4_valid = true;
}

// F in FP64 for the NB_F64 kernel: its reads then need no conversion, each
// of which costs an FP64-pipe instruction (2x the table's memory; skipped,
// and the kernel converts, if that allocation fails)
static void ensure_f64_table(nb_sim *s) {
  if (s->F64_valid || s->precision != NB_F64) return;
  const long long n = (long long)s->hn[0] * s->hn[1] * s->hn[2];
  if (s->d_F64t.ensure((size_t)n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (nbgb::build_f64_table((const float *)s->d_F.p, n,
                            (double *)s->d_F64t.p, s->stream) == cudaSuccess)
    s->F64_valid = true;
}

// the tricubic polynomial of every table cell (64 floats per cell) for the
// warp-per-pixel kernel; skipped above 2 GB, for an axis longer than 1000
// nodes, or if the allocation fails
static void ensure_cell_polynomials(nb_sim *s) {
  if (s->C4_valid || s->interp != NB_INTERP_TRICUBIC ||
      s->precision != NB_MIXED)
    return;
  if (s->hn[0] < 4 || s->hn[1] < 4 || s->hn[2] < 4) return;
  // the warp kernel packs a table index into 10 bits per axis
  if (s->hn[0] > 1000 || s->hn[1] > 1000 || s->hn[2] > 1000) return;
  size_t cells = (size_t)(s->hn[0] - 3) * (s->hn[1] - 3) * (s->hn[2] - 3);
  size_t bytes = cells * 16 * sizeof(float4);
  if (bytes > (size_t)2 << 30) return;
  if (s->d_C4.ensure(bytes) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (nbgb::build_cell_polynomials((const float *)s->d_F.p, s->hn,
                                   (float4 *)s->d_C4.p,
                                   s->stream) == cudaSuccess)
    s->C4_valid = true;
}

static int launch(nb_sim *s, const long long *dev_list, long long n_list) {
  if (!s->have_crystal || !s->have_beam || !s->have_det || !s->have_F)
    return fail(s, NB_ESTATE, "crystal, beam and detector must be set first");
  int rc = upload_tables(s);
  if (rc != NB_OK) return rc;
  ensure_sliding_table(s);
  ensure_f64_table(s);
  SpotArgs a;
  fill_args(s, a);
  a.pixlist = dev_list;
  a.n_list = n_list;
  size_t smem_need =
      s->precision == NB_F64
          ? (size_t)(a.PM * 9 + a.S * nbgb::SRC64_STRIDE) * sizeof(double)
          : (size_t)(2 * a.PM * 9 + a.S * nbgb::SRC32_STRIDE) *
                sizeof(float);
  if (smem_need > 200 * 1024)
    return fail(s, NB_EINVAL,
                "phi x mosaic and source tables exceed 200 KB of shared "
                "memory");
  // the sinc fast path stages 8 more floats per pair of sources; where
  // they do not fit as well, the kernels take the general path
  if (a.srcq &&
      smem_need + (size_t)8 * ((a.S + 1) / 2) * sizeof(float) > 200 * 1024) {
    a.srcq = nullptr;
    a.sinc_qG = 0.f;
  }
  // counters: [0] evaluated terms, [1..3] the warp kernel's pairs,
  // intervals and source blocks
  cudaError_t e = s->d_stats.ensure(4 * sizeof(unsigned long long));
  if (e != cudaSuccess) return fail(s, NB_ENOMEM, "statistics counters");
  e = cudaMemsetAsync(s->d_stats.p, 0, 4 * sizeof(unsigned long long),
                      s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "statistics reset");
  a.stats = (unsigned long long *)s->d_stats.p;
  a.wstats = s->count_work ? a.stats + 1 : nullptr;
  long long pix = dev_list ? n_list : s->npix;
  s->last_pixel_steps = pix * (long long)s->os * s->os * s->T * s->n_src *
                        s->n_mosaic * s->n_phi;
  s->last_pixels = pix;
  // one warp per pixel pays off where the scattered terms are expensive
  // (tricubic lookups) and a pixel has enough items to fill the lanes
  bool auto_warp = a.interp == NB_INTERP_TRICUBIC &&
                   (long long)a.os * a.os * a.T * a.PM >= 8;
  bool warp_variant =
      s->precision == NB_MIXED && nbgb::split_supported(a) &&
      (s->variant == NB_VARIANT_WARP ||
       (s->variant == NB_VARIANT_AUTO && auto_warp));
  s->last_warp = warp_variant && s->precision != NB_F64;
  s->last_counted = s->count_work;
  if (s->precision == NB_F64) {
    e = nbgb::launch_spots_f64(a, s->stream);
  } else if (warp_variant) {
    ensure_cell_polynomials(s);
    a.C4 = s->C4_valid ? (const float4 *)s->d_C4.p : nullptr;
    e = s->d_work.ensure(sizeof(unsigned long long));
    if (e != cudaSuccess) return fail(s, NB_ENOMEM, "work counter");
    e = cudaMemsetAsync(s->d_work.p, 0, sizeof(unsigned long long),
                        s->stream);
    if (e == cudaSuccess)
      e = nbgb::launch_spots_split(a, (unsigned long long *)s->d_work.p,
                                   s->sm_count, s->stream);
  } else {
    e = nbgb::launch_spots_mixed(a, s->precision, s->stream);
  }
  if (e != cudaSuccess) return cuda_fail(s, e, "spots launch");
  return read_check(s);
}

int nb_add_spots(nb_sim *s) {
  nbgb::NvtxRange nvtx_("nb_add_spots");
  if (!s) return NB_EINVAL;
  DeviceGuard g(s->device);
  return launch(s, nullptr, 0);
}

int nb_add_spots_pixels(nb_sim *s, const long long *pixels,
                        long long n_pix) {
  nbgb::NvtxRange nvtx_("nb_add_spots_pixels");
  if (!s) return NB_EINVAL;
  if (n_pix < 0 || (n_pix > 0 && !pixels))
    return fail(s, NB_EINVAL, "pixel list");
  if (!s->have_det) return fail(s, NB_ESTATE, "detector not set");
  for (long long i = 0; i < n_pix; ++i)
    if (pixels[i] < 0 || pixels[i] >= s->npix)
      return fail(s, NB_EINVAL, "pixel index out of range");
  if (n_pix == 0) return NB_OK;
  DeviceGuard g(s->device);
  // the list buffer may still be read by an earlier launch on the stream
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "stream sync");
  e = s->d_list.ensure((size_t)n_pix * sizeof(long long));
  if (e != cudaSuccess) return fail(s, NB_ENOMEM, "pixel list");
  e = cudaMemcpyAsync(s->d_list.p, pixels, (size_t)n_pix * sizeof(long long),
                      cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "pixel list upload");
  return launch(s, (const long long *)s->d_list.p, n_pix);
}

int nb_zero_image(nb_sim *s) {
  nbgb::NvtxRange nvtx_("nb_zero_image");
  if (!s) return NB_EINVAL;
  if (!s->have_det) return fail(s, NB_ESTATE, "detector not set");
  DeviceGuard g(s->device);
  cudaError_t e = cudaMemsetAsync(s->d_image.p, 0,
                                  (size_t)s->npix * sizeof(double), s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "image clear");
  return NB_OK;
}

__global__ void nb_to_f32_kernel(const double *src, float *dst, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += stride) dst[i] = (float)src[i];
}

int nb_get_image(nb_sim *s, void *dst, size_t n_elems, int dtype,
                 int on_device) {
  nbgb::NvtxRange nvtx_("nb_get_image");
  if (!s) return NB_EINVAL;
  if (!dst) return fail(s, NB_EINVAL, "dst NULL");
  if (!s->have_det) return fail(s, NB_ESTATE, "detector not set");
  if ((long long)n_elems != s->npix)
    return fail(s, NB_EINVAL, "n_elems differs from the pixel count");
  if (dtype != NB_DTYPE_F32 && dtype != NB_DTYPE_F64)
    return fail(s, NB_EINVAL, "bad dtype");
  DeviceGuard g(s->device);
  cudaError_t e;
  size_t n = n_elems;
  if (dtype == NB_DTYPE_F64) {
    e = cudaMemcpyAsync(dst, s->d_image.p, n * 8,
                        on_device ? cudaMemcpyDeviceToDevice
                                  : cudaMemcpyDeviceToHost,
                        s->stream);
  } else {
    float *target = (float *)dst;
    if (!on_device) {
      e = s->d_tmp.ensure(n * 4);
      if (e != cudaSuccess) return fail(s, NB_ENOMEM, "conversion buffer");
      target = (float *)s->d_tmp.p;
    }
    nb_to_f32_kernel<<<1216, 256, 0, s->stream>>>((const double *)s->d_image.p,
                                                  target, (long long)n);
    e = cudaGetLastError();
    if (e == cudaSuccess && !on_device)
      e = cudaMemcpyAsync(dst, s->d_tmp.p, n * 4, cudaMemcpyDeviceToHost,
                          s->stream);
  }
  if (e != cudaSuccess) return cuda_fail(s, e, "image copy");
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "image copy sync");
  return NB_OK;
}

const double *nb_image_device_ptr(const nb_sim *s) {
  return (s && s->have_det) ? (const double *)s->d_image.p : nullptr;
}

int nb_adjoint(nb_sim *s, const double *dLdI, double grad[10],
               double *gradF) {
  nbgb::NvtxRange nvtx_("nb_adjoint");
  if (!s) return NB_EINVAL;
  if (!dLdI || !grad) return fail(s, NB_EINVAL, "NULL dLdI / grad");
  if (!s->have_crystal || !s->have_beam || !s->have_det || !s->have_F)
    return fail(s, NB_ESTATE, "crystal, beam and detector must be set first");
  if (!s->have_params)
    return fail(s, NB_ESTATE, "nb_set_crystal_params must come first");
  if (s->precision != NB_MIXED || s->shape != NB_SHAPE_GAUSS)
    return fail(s, NB_EINVAL,
                "the adjoint needs NB_MIXED and a Gaussian shape");
  DeviceGuard g(s->device);
  int rc = upload_tables(s);
  if (rc != NB_OK) return rc;
  if (s->has_div)
    return fail(s, NB_EINVAL, "the adjoint needs one source direction");
  ensure_cell_polynomials(s);  // tricubic value and gradient per cell
  SpotArgs a;
  fill_args(s, a);
  if (nbgb::adjoint_smem_bytes(a, a.interp == NB_INTERP_TRICUBIC && gradF) >
      200 * 1024)
    return fail(s, NB_EINVAL, "tables exceed 200 KB of shared memory");
  long long blocks = nbgb::adjoint_blocks(a);
  cudaError_t e = s->d_part.ensure((size_t)(blocks + 1) * 10 * sizeof(double));
  if (e == cudaSuccess) e = s->d_grad.ensure(16 * sizeof(double));
  if (e != cudaSuccess) return fail(s, NB_ENOMEM, "gradient scratch");
  double kc = nbgb::kElectronRadius * nbgb::kElectronRadius * s->fluence /
              ((double)s->os * s->os * s->n_mosaic * s->n_phi);
  e = nbgb::launch_adjoint(a, (const float *)s->d_dax.p, dLdI, gradF,
                           (double *)s->d_part.p, kc, s->scale,
                           (double *)s->d_grad.p, s->sm_count, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(grad, s->d_grad.p, 10 * sizeof(double),
                        cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "adjoint");
  return read_check(s);
}

int nb_poisson_loss(nb_sim *s, const double *y, double bkg, double *dLdI,
                    double *loss) {
  nbgb::NvtxRange nvtx_("nb_poisson_loss");
  if (!s) return NB_EINVAL;
  if (!y || !dLdI || !loss) return fail(s, NB_EINVAL, "NULL argument");
  if (!s->have_det) return fail(s, NB_ESTATE, "detector not set");
  if (!(bkg > 0) || !std::isfinite(bkg))
    return fail(s, NB_EINVAL, "bkg must be positive");
  DeviceGuard g(s->device);
  int blocks = nbgb::loss_blocks(s->npix);
  cudaError_t e = s->d_part.ensure((size_t)(blocks + 1) * 10 * sizeof(double));
  if (e == cudaSuccess) e = s->d_grad.ensure(16 * sizeof(double));
  if (e != cudaSuccess) return fail(s, NB_ENOMEM, "loss scratch");
  e = nbgb::launch_poisson_loss((const double *)s->d_image.p, y, s->npix, bkg,
                                dLdI, (double *)s->d_part.p,
                                (double *)s->d_grad.p, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(loss, s->d_grad.p, sizeof(double),
                        cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "loss");
  return NB_OK;
}

int nb_set_option(nb_sim *s, int key, long long value) {
  if (!s) return NB_EINVAL;
  if (key == NB_OPT_VARIANT) {
    if (value < NB_VARIANT_AUTO || value > NB_VARIANT_WARP)
      return fail(s, NB_EINVAL, "bad variant");
    s->variant = (int)value;
    return NB_OK;
  }
  if (key == NB_OPT_COUNT_WORK) {
    if (value != 0 && value != 1) return fail(s, NB_EINVAL, "bad value");
    s->count_work = value != 0;
    return NB_OK;
  }
  if (key == NB_OPT_FAIL_ALLOCS) {
    if (value < 0) return fail(s, NB_EINVAL, "bad value");
    g_fail_allocs.store(value);
    return NB_OK;
  }
  return fail(s, NB_EINVAL, "unknown option");
}

int nb_get_stats(nb_sim *s, long long *evaluated_terms,
                 long long *pixel_steps) {
  nbgb::NvtxRange nvtx_("nb_get_stats");
  if (!s) return NB_EINVAL;
  if (!evaluated_terms || !pixel_steps)
    return fail(s, NB_EINVAL, "NULL output");
  *evaluated_terms = 0;
  *pixel_steps = s->last_pixel_steps;
  if (!s->d_stats.p) return NB_OK;
  DeviceGuard g(s->device);
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, s->d_stats.p, sizeof v,
                                  cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "statistics read");
  *evaluated_terms = (long long)v;
  return NB_OK;
}

int nb_get_work(nb_sim *s, long long *counts, int n_counts) {
  nbgb::NvtxRange nvtx_("nb_get_work");
  if (!s) return NB_EINVAL;
  if (!counts || n_counts < 1) return fail(s, NB_EINVAL, "NULL output");
  long long v[NB_WORK_N] = {0};
  v[NB_WORK_PIXEL_STEPS] = s->last_pixel_steps;
  const long long units = s->last_pixels * (long long)s->os * s->os * s->T;
  v[NB_WORK_UNITS] = units;
  v[NB_WORK_ITEMS] = units * s->n_mosaic * s->n_phi;
  if (s->d_stats.p) {
    DeviceGuard g(s->device);
    unsigned long long c[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(c, s->d_stats.p, sizeof c,
                                    cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "statistics read");
    if (s->precision == NB_F64) {
      // every step is tested and evaluated
      v[NB_WORK_PAIRS] = v[NB_WORK_TERMS] = s->last_pixel_steps;
    } else {
      v[NB_WORK_TERMS] = (long long)c[0];
      if (!s->last_warp) {
        // the thread-per-pixel kernels test every step
        v[NB_WORK_PAIRS] = s->last_pixel_steps;
      } else if (s->last_counted) {
        v[NB_WORK_PAIRS] = (long long)c[1];
        v[NB_WORK_INTERVALS] = (long long)c[2];
        v[NB_WORK_BLOCKS] = (long long)c[3];
      } else {
        v[NB_WORK_PAIRS] = v[NB_WORK_INTERVALS] = v[NB_WORK_BLOCKS] = -1;
      }
    }
  }
  for (int i = 0; i < n_counts; ++i) counts[i] = i < NB_WORK_N ? v[i] : 0;
  return NB_OK;
}

int nb_set_background(nb_sim *s, const double *stol, const double *F,
                      int n_knots, double n_molecules) {
  nbgb::NvtxRange nvtx_("nb_set_background");
  if (!s) return NB_EINVAL;
  if (!stol || !F) return fail(s, NB_EINVAL, "NULL background table");
  if (n_knots < 2 || n_knots > nbgb::kMaxKnots)
    return fail(s, NB_EINVAL, "need 2 <= n_knots <= 4096");
  for (int j = 0; j < n_knots; ++j) {
    if (!std::isfinite(stol[j]) || !std::isfinite(F[j]))
      return fail(s, NB_EINVAL, "background table not finite");
    if (j > 0 && !(stol[j] > stol[j - 1]))
      return fail(s, NB_EINVAL, "background knots must increase strictly");
  }
  if (!(n_molecules >= 0) || !std::isfinite(n_molecules))
    return fail(s, NB_EINVAL, "n_molecules");
  s->bg_stol.assign(stol, stol + n_knots);
  s->bg_F.assign(F, F + n_knots);
  s->bg_nmol = n_molecules;
  s->have_bg = true;
  return NB_OK;
}

int nb_add_background(nb_sim *s) {
  nbgb::NvtxRange nvtx_("nb_add_background");
  if (!s) return NB_EINVAL;
  if (!s->have_beam || !s->have_det || !s->have_bg)
    return fail(s, NB_ESTATE,
                "beam, detector and background table must be set first");
  DeviceGuard g(s->device);
  const int S = s->n_src, n = (int)s->bg_stol.size();
  // group the sources (already in ascending 1/lambda) by direction; the
  // order inside a group stays ascending
  std::vector<int> order, rng;
  std::vector<double> grp;
  std::vector<char> used(S, 0);
  for (int k = 0; k < S; ++k) {
    if (used[k]) continue;
    const double *dk = s->dirs.data() + 3 * k;
    int first = (int)order.size();
    for (int l = k; l < S; ++l) {
      const double *dl = s->dirs.data() + 3 * l;
      if (!used[l] && dl[0] == dk[0] && dl[1] == dk[1] && dl[2] == dk[2]) {
        used[l] = 1;
        order.push_back(l);
      }
    }
    double ep[3], bp[3];
    pol_basis(dk, s->evec, ep, bp);
    for (int c = 0; c < 3; ++c) grp.push_back(dk[c]);
    for (int c = 0; c < 3; ++c) grp.push_back(ep[c]);
    for (int c = 0; c < 3; ++c) grp.push_back(bp[c]);
    rng.push_back(first);
    rng.push_back((int)order.size() - first);
  }
  const int G = (int)rng.size() / 2;
  const bool f64 = s->precision == NB_F64;
  // one double blob: groups, then (F64) knots and sources; one float blob
  std::vector<double> b64(grp);
  std::vector<float> b32;
  if (f64) {
    for (int j = 0; j < n; ++j) {
      b64.push_back(s->bg_stol[j]);
      b64.push_back(s->bg_F[j]);
    }
    for (int k : order) {
      b64.push_back(1.0 / s->lam[k]);
      b64.push_back(s->w[k]);
    }
  } else {
    for (int j = 0; j < n; ++j) {
      double slope = j + 1 < n ? (s->bg_F[j + 1] - s->bg_F[j]) /
                                     (s->bg_stol[j + 1] - s->bg_stol[j])
                               : 0.0;
      b32.push_back((float)s->bg_stol[j]);
      b32.push_back((float)s->bg_F[j]);
      b32.push_back((float)slope);
    }
    for (int k : order) {
      b32.push_back((float)(1.0 / s->lam[k]));
      b32.push_back((float)s->w[k]);
    }
  }
  cudaError_t e;
  if ((e = s->d_bg64.ensure(b64.size() * 8)) != cudaSuccess ||
      (e = s->d_bg32.ensure(std::max<size_t>(b32.size(), 1) * 4)) !=
          cudaSuccess ||
      (e = s->d_bgrng.ensure(rng.size() * sizeof(int))) != cudaSuccess)
    return fail(s, NB_ENOMEM, "background tables");
  cudaMemcpyAsync(s->d_bg64.p, b64.data(), b64.size() * 8,
                  cudaMemcpyHostToDevice, s->stream);
  if (!b32.empty())
    cudaMemcpyAsync(s->d_bg32.p, b32.data(), b32.size() * 4,
                    cudaMemcpyHostToDevice, s->stream);
  cudaMemcpyAsync(s->d_bgrng.p, rng.data(), rng.size() * sizeof(int),
                  cudaMemcpyHostToDevice, s->stream);
  nbgb::BgArgs b;
  std::memset(&b, 0, sizeof b);
  SpotArgs &a = b.geo;
  a.check = (unsigned long long *)s->d_check.p;  // NB_CHECK builds only
  a.panels = (const DevPanel *)s->d_panels.p;
  a.n_panels = (int)s->panels.size();
  a.n_tiles = s->n_tiles;
  a.npix = s->npix;
  a.os = s->os;
  a.T = s->T;
  a.dt = s->thick > 0 ? s->thick / s->T : 0.0;
  a.thickness = s->thick;
  a.atten = s->atten;
  a.S = S;
  a.kahn64 = s->kahn;
  a.image = (double *)s->d_image.p;
  b.n_knots = n;
  b.n_groups = G;
  const double *d64 = (const double *)s->d_bg64.p;
  b.grp64 = d64;
  b.knots64 = d64 + 9 * G;
  b.src64 = d64 + 9 * G + 2 * n;
  b.knots32 = (const float *)s->d_bg32.p;
  b.src32 = b.knots32 + 3 * n;
  b.grp_range = (const int *)s->d_bgrng.p;
  b.prefactor = nbgb::kElectronRadius * nbgb::kElectronRadius * s->fluence *
                s->bg_nmol / ((double)s->os * s->os);
  if (nbgb::background_smem_bytes(b, f64) > 200 * 1024)
    return fail(s, NB_EINVAL,
                "background tables exceed 200 KB of shared memory");
  e = nbgb::launch_background(b, f64, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "background launch");
  // the pageable copies above are staged before the launch returns
  return read_check(s);
}

int nb_synchronize(nb_sim *s) {
  nbgb::NvtxRange nvtx_("nb_synchronize");
  if (!s) return NB_EINVAL;
  DeviceGuard g(s->device);
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "synchronize");
  return NB_OK;
}

}  // extern "C"
