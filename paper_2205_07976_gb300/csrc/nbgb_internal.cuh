// nbgb_internal.cuh -- kernel-side data layout and helpers of libnbgb.
//
// Layout in HBM (all device buffers owned by one nb_sim handle):
//   panels   DevPanel[n_panels]            geometry + pixel/tile offsets
//   ax64     double[PM][9]                 U_m R_phi (a,b,c)_lab, PM = Phi*M
//   axh/axl  float[PM][9]                  double-float split of ax64
//   src64    double[S][SRC64_STRIDE]       lambda, w, dir, E', B'
//   src32    float [S][SRC32_STRIDE]       delta_lo, w, delta_hi, dir, E', B'
//   divh/l   float[PM][S][3]               divergence term (only if sources
//                                           do not share one direction)
//   F        float[nh][nk][nl]             structure factors, l fastest
//   image    double[npix]                  resident accumulator
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <vector>

#ifndef NB_CHECK
#define NB_CHECK 0
#endif

namespace nbgb {

// Bounds checks of the kernels' table and image indexing, compiled in only
// with -DNB_CHECK=1 (the debug build; `_build.build(variant="check")`).  A
// failed check records its site and index in a device word (the first one
// wins) and the access uses index 0 instead, so nothing faults; the host
// reads the word after each launch and the call returns NB_ECUDA with the
// site and index in nb_last_error.  Without NB_CHECK the index passes
// through unchanged.
enum {
  NB_SITE_F = 1,        // structure-factor entry (nearest lookup)
  NB_SITE_STENCIL = 2,  // last entry of a 4x4x4 tricubic stencil
  NB_SITE_CELL = 3,     // cell polynomial
  NB_SITE_IMAGE = 4,    // image pixel
  NB_SITE_SOURCE = 5,   // source row
  NB_SITE_GRADF = 6,    // structure-factor gradient entry
  NB_SITE_KNOT = 7      // background knot
};

__device__ __forceinline__ long long nb_idx(unsigned long long *word, int site,
                                           long long i, long long n) {
#if NB_CHECK
  if ((unsigned long long)i >= (unsigned long long)n) {
    if (word)
      atomicCAS(word, 0ull,
                (1ull << 63) | ((unsigned long long)site << 56) |
                    ((unsigned long long)i & ((1ull << 56) - 1)));
    return 0;
  }
#else
  (void)word;
  (void)site;
  (void)n;
#endif
  return i;
}

// An NVTX range named after a C-ABI call, pushed for the call's duration:
// profilers that attach an NVTX tool show the library's calls on the host
// timeline (without a tool the push and pop cost a branch).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr double kElectronRadius = 2.8179403262e-15;  // m, CODATA 2018
constexpr int kTileF = 16;                            // pixels per tile, fast
constexpr int kTileS = 8;                             // pixels per tile, slow
constexpr int kTileThreads = kTileF * kTileS;
constexpr int kMaxPM = 2048;
constexpr int kMaxSrc = 1024;
// Gaussian terms with sum N^2 f^2 / 0.63 above this are skipped: their
// F_latt^2 / (Na Nb Nc)^2 = exp(-2 * 44) < FLT_MIN, i.e. they vanish in the
// FP32 evaluation anyway.
constexpr float kGaussCut = 44.0f;

enum { SRC64_LAM = 0, SRC64_W = 1, SRC64_DIR = 2, SRC64_E = 5, SRC64_B = 8,
       SRC64_STRIDE = 11 };
// (delta_lo, w) first: the warp kernel reads the pair as one float2
enum { SRC32_DL = 0, SRC32_W = 1, SRC32_DH = 2, SRC32_DIR = 3, SRC32_E = 6,
       SRC32_B = 9, SRC32_STRIDE = 12 };

struct DevPanel {
  double origin[3];
  double fdir[3];
  double sdir[3];
  double ndir[3];
  double px;
  // the same vectors as double-float pairs (hi, lo) for the FP32 kernels'
  // geometry (panel_ff fills them)
  float ffo[3][2], fff[3][2], ffs[3][2], ffn[3][2], ffpx[2];
  long long pix0;  // global index of pixel (0, 0)
  int nfast, nslow;
  int tile0;       // first tile of this panel in the tiled launch
  int tiles_f;     // tiles along fast
  int tiles;       // tiles of this panel
  int pad;
};

struct SpotArgs {
  // detector
  const DevPanel *panels;
  int n_panels;
  int n_tiles;
  long long npix;
  const long long *pixlist;  // non-null: launch over this pixel list
  long long n_list;
  int os, T;
  double dt, thickness, atten;
  // crystal
  int PM;
  const double *ax64;
  const float *axh, *axl;
  double N64[3];
  float N[3];
  float N6;  // (Na Nb Nc)^2
  int shape, interp;
  const float *F;
  // optional copy of F in FP64 for the NB_F64 kernel (null: each read
  // converts F's float)
  const double *F64t;
  // optional copy of F for tricubic lookups: F4[i][j][l] holds
  // F[i][j][l..l+3] (zero past the end), one 16-byte load per stencil row
  const float4 *F4;
  // optional tricubic cell polynomials: for the cell whose 4x4x4 stencil
  // starts at table node (i, j, k), 16 float4 = the 64 monomial
  // coefficients C[a][b][c] of x^a y^b z^c, x in [0, 1) from node + 1;
  // float4 2 (4 P + b) holds C[2P][b][3], C[2P+1][b][3], C[2P][b][2],
  // C[2P+1][b][2] and the next one the same for c = 1 and c = 0
  const float4 *C4;
  int hmin[3], hn[3];
  float defF;
  double defF64;
  // beam
  int S;
  const double *src64;
  const float *src32;
  double u0;
  float u0h, u0l;
  double i0[3];  // direction of source 0 (all sources, unless has_div)
  float i0ff[3][2];  // i0 and dt as double-float pairs, and FP32 copies of
  float dtff[2];     // e0, b0 and the attenuation length (args_ff)
  float e0f[3], b0f[3], attenf;
  double e0[3], b0[3];
  float kahn;
  double kahn64;
  int has_div;
  const float *divh, *divl;
  // sinc fast path of NB_MIXED: per source delta split on a fixed grid qD
  // (srcq: per pair of sources (delta on the grid x2, the rest x2, w x2,
  // delta x2)), and the grid qG of the items' G, with qG qD = 2^-21;
  // sinc_qG = 0: no fast path
  const float *srcq;
  float sinc_qG;
  float sinc_dq[2];  // the least and the largest delta on the grid qD
  double prefactor;  // r_e^2 fluence scale / (os^2 M Phi)
  double *image;
  // statistics of the launch: [0] terms evaluated (the FP32 forms skip
  // Gaussian terms that underflow); null to skip counting
  unsigned long long *stats;
  // work the warp-per-pixel kernel performs besides the terms: [0]
  // (interval, source) pairs tested against the cut, [1] lattice-point
  // intervals solved, [2] source blocks tested; null to skip counting (the
  // kernel is then instantiated without the counters)
  unsigned long long *wstats;
  // NB_CHECK builds: the word a failed bounds check writes (null: none)
  unsigned long long *check;
};

__device__ __forceinline__ long long table_size(const SpotArgs &a) {
  return (long long)a.hn[0] * a.hn[1] * a.hn[2];
}
__device__ __forceinline__ long long cell_count(const SpotArgs &a) {
  return (long long)(a.hn[0] - 3) * (a.hn[1] - 3) * (a.hn[2] - 3);
}
// offset in F of row (i, j) of the 4x4x4 stencil that starts at fl - 1
// (its 4 entries checked in NB_CHECK builds)
__device__ __forceinline__ long long stencil_row(const SpotArgs &a,
                                                 const int fl[3], int i,
                                                 int j) {
  const long long off =
      ((long long)(fl[0] - 1 + i) * a.hn[1] + (fl[1] - 1 + j)) * a.hn[2] +
      (fl[2] - 1);
  return nb_idx(a.check, NB_SITE_STENCIL, off + 3, table_size(a)) == off + 3
             ? off
             : 0;
}

// host: v as a double-float pair, hi = v rounded to FP32, lo the rest
inline void split_ff_host(double v, float ff[2]) {
  ff[0] = (float)v;
  ff[1] = (float)(v - (double)ff[0]);
}

// host: fills the double-float copies of a panel's vectors
inline void panel_ff(DevPanel &d) {
  for (int c = 0; c < 3; ++c) {
    split_ff_host(d.origin[c], d.ffo[c]);
    split_ff_host(d.fdir[c], d.fff[c]);
    split_ff_host(d.sdir[c], d.ffs[c]);
    split_ff_host(d.ndir[c], d.ffn[c]);
  }
  split_ff_host(d.px, d.ffpx);
}

// host: fills the double-float and FP32 copies of the beam vectors, the
// layer thickness and the attenuation length in a filled SpotArgs
inline void args_ff(SpotArgs &a) {
  for (int c = 0; c < 3; ++c) {
    split_ff_host(a.i0[c], a.i0ff[c]);
    a.e0f[c] = (float)a.e0[c];
    a.b0f[c] = (float)a.b0[c];
  }
  split_ff_host(a.dt, a.dtff);
  a.attenf = (float)a.atten;
}

// adds v of every active lane to *ctr with one atomic per converged group
__device__ __forceinline__ void warp_count(unsigned long long *ctr,
                                           unsigned v) {
  unsigned mask = __activemask();
  unsigned tot = __reduce_add_sync(mask, v);
  if ((threadIdx.x & 31) == __ffs(mask) - 1)
    atomicAdd(ctr, (unsigned long long)tot);
}

// ---------------------------------------------------------------- mapping

__device__ __forceinline__ int panel_of_tile(const SpotArgs &a, int tile) {
  int lo = 0, hi = a.n_panels - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (a.panels[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int panel_of_pixel(const SpotArgs &a,
                                              long long g) {
  int lo = 0, hi = a.n_panels - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (a.panels[mid].pix0 <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Pixel handled by (block, thread): a 16x8 tile per block, or one entry of
// the pixel list.  Returns false for threads past the panel edge.
__device__ __forceinline__ bool map_pixel(const SpotArgs &a, long long item,
                                          int lane_in_tile, long long &gp,
                                          int &q, int &s, int &f) {
  if (a.pixlist) {
    if (item >= a.n_list) return false;
    gp = a.pixlist[item];
    q = panel_of_pixel(a, gp);
    long long local = gp - a.panels[q].pix0;
    int nf = a.panels[q].nfast;
    s = (int)(local / nf);
    f = (int)(local - (long long)s * nf);
    return true;
  }
  int tile = (int)item;
  if (tile >= a.n_tiles) return false;
  q = panel_of_tile(a, tile);
  const DevPanel &P = a.panels[q];
  int t = tile - P.tile0;
  int ts = t / P.tiles_f, tf = t - ts * P.tiles_f;
  s = ts * kTileS + lane_in_tile / kTileF;
  f = tf * kTileF + lane_in_tile % kTileF;
  if (s >= P.nslow || f >= P.nfast) return false;
  gp = P.pix0 + (long long)s * P.nfast + f;
  return true;
}

// ------------------------------------------------- error-free FP32 steps
// (Dekker / Knuth transformations; the _rn intrinsics keep the compiler
// from contracting them into FMAs)

__device__ __forceinline__ void two_sum(float a, float b, float &s,
                                        float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s,
                                             float &e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p,
                                         float &e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// Kahan-compensated FP32 accumulation
struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const {
    return (double)s - (double)c;
  }
};

// sin(pi x) for |x| <= ~0.55: x * p(x^2), p the degree-5 least-squares fit
// of sin(pi x)/x in x^2 at 400 Chebyshev nodes of [0, 0.56] (max relative
// error 1e-10 in exact arithmetic, ~2 ulp evaluated in FP32).
__device__ __forceinline__ float sinpi_reduced(float x) {
  float t = x * x;
  float p = -6.941131045e-03f;
  p = fmaf(p, t, 8.199509639e-02f);
  p = fmaf(p, t, -5.992401060e-01f);
  p = fmaf(p, t, 2.550162271e+00f);
  p = fmaf(p, t, -5.167712735e+00f);
  p = fmaf(p, t, 3.141592653e+00f);
  return x * p;
}

// 4-point Lagrange weights for nodes -1, 0, 1, 2 at x in [0, 1]
template <typename T>
__device__ __forceinline__ void lagrange4(T x, T w[4]) {
  T xm1 = x - T(1), xm2 = x - T(2), xp1 = x + T(1);
  T a = x * xm1;      // x (x-1)
  T b = xp1 * xm2;    // (x+1)(x-2)
  w[0] = -a * xm2 * T(1.0 / 6.0);
  w[1] = b * xm1 * T(0.5);
  w[2] = -b * x * T(0.5);
  w[3] = a * xp1 * T(1.0 / 6.0);
}

// host-side table builders shared by nb_sim and nb_server
void sort_sources(std::vector<double> &dirs, std::vector<double> &lam,
                  std::vector<double> &w);
double source_u0(const double *lam, int S);
void shot_tables_f32(const std::vector<double> &ax, const double *lam,
                     const double *w, const double *dirs, int S,
                     const double *evec, double u0, bool plain_f32,
                     std::vector<float> &axh, std::vector<float> &axl,
                     std::vector<float> &src32);
void rotated_axes_table(const double *lab, const double *umats, int n_mosaic,
                        int n_phi, double phi0_deg, double phistep_deg,
                        const double *spindle, std::vector<double> &ax);

cudaError_t launch_spots_f64(const SpotArgs &a, cudaStream_t st);
cudaError_t build_f64_table(const float *F, long long n, double *F64t,
                            cudaStream_t st);
cudaError_t build_sliding_table(const float *F, const int hn[3], float4 *F4,
                                cudaStream_t st);
cudaError_t build_cell_polynomials(const float *F, const int hn[3], float4 *C4,
                                   cudaStream_t st);
size_t adjoint_smem_bytes(const SpotArgs &a, bool f_cache);
long long adjoint_blocks(const SpotArgs &a);
int loss_blocks(long long n);
cudaError_t launch_adjoint(const SpotArgs &a, const float *dax,
                           const double *dLdI, double *gradF,
                           double *partials, double kc, double scale,
                           double *grad_out, int sm_count, cudaStream_t st);
cudaError_t launch_poisson_loss(const double *img, const double *y,
                                long long n, double bkg, double *dLdI,
                                double *partials, double *loss_out,
                                cudaStream_t st);
size_t split_smem_bytes(const SpotArgs &a);
bool split_supported(const SpotArgs &a);
cudaError_t launch_spots_split(const SpotArgs &a, unsigned long long *work,
                               int sm_count, cudaStream_t st);
size_t serve_warp_smem_bytes();
cudaError_t launch_spots_mixed(const SpotArgs &a, int precision,
                               cudaStream_t st);

// amorphous background: the detector and beam fields of SpotArgs plus the
// scattering table and the sources grouped by direction (ascending 1/lambda
// within a group)
struct BgArgs {
  SpotArgs geo;
  int n_knots, n_groups;
  const double *knots64;  // [n][2] stol, F
  const float *knots32;   // [n][3] stol, F, slope to the next knot
  const double *grp64;    // [G][9] direction, E', B'
  const int *grp_range;   // [G][2] first source, count
  const double *src64;    // [S][2] 1/lambda, w (grouped order)
  const float *src32;     // [S][2]
  double prefactor;       // r_e^2 fluence n_mol / os^2
};
constexpr int kMaxKnots = 4096;
size_t background_smem_bytes(const BgArgs &b, bool f64);
cudaError_t launch_background(const BgArgs &b, bool f64, cudaStream_t st);

}  // namespace nbgb
