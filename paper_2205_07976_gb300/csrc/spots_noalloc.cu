// spots_noalloc.cu -- nb_add_spots_noalloc: the warp-per-pixel FP32-mixed
// Bragg-spot kernel run without any allocation by the library.
//
// Who needs it: code that must not call cudaMalloc at all -- work queued
// while another component owns every allocation (a caller's own memory
// pool or arena), code inside a region where allocating would synchronise
// the device, or a plug-in whose host forbids device allocation.  The
// regular entry points allocate the handle's tables in nb_set_*; this one
// takes every input and the output as caller-owned device memory.
//
// Its scratch (the converted tables the kernel stages, one panel record
// and two counters) lives in the file-scope array below: kScratchBytes on
// every GPU that loads the library, held until the process exits.  All
// calls share it, so calls whose work overlaps on the GPU (different
// streams, or different host threads) race; serialise them.  Every call
// rewrites the tables and zeroes the counters before the kernel runs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/nbgb.h"
#include "nbgb_internal.cuh"

namespace nbgb {

namespace {

constexpr int kNoAllocMaxPM = kMaxPM;    // phi steps x mosaic domains
constexpr int kNoAllocMaxSrc = kMaxSrc;  // sources
// tables: axes hi/lo [PM][9] + sources [S][SRC32_STRIDE] floats, then one
// DevPanel, then 2 counters (work, evaluated terms)
constexpr size_t kTableFloats =
    (size_t)kNoAllocMaxPM * 18 + (size_t)kNoAllocMaxSrc * SRC32_STRIDE;
constexpr size_t kPanelOffset = ((kTableFloats * 4 + 255) / 256) * 256;
constexpr size_t kCounterOffset =
    kPanelOffset + ((sizeof(DevPanel) + 255) / 256) * 256;
constexpr size_t kScratchBytes = kCounterOffset + 256;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

struct TableArgs {
  const double *axes;  // [PM][9]
  const double *lam;   // [S]
  const double *w;     // [S]
  int PM, S;
  float dir[3], ep[3], bp[3];
  DevPanel panel;
  float *axh, *axl, *src32;
  DevPanel *panel_out;
  unsigned long long *counters;
  double *u0_out;  // u0 written here for the spots launch
};

// One block: u0 = centre of the 1/lambda range, then the double-float
// tables in the layout the warp-per-pixel kernel stages.
__global__ void noalloc_tables_kernel(TableArgs t) {
  __shared__ double s_min[256], s_max[256];
  double mn = 1e300, mx = -1e300;
  for (int k = threadIdx.x; k < t.S; k += blockDim.x) {
    double u = 1.0 / t.lam[k];
    mn = fmin(mn, u);
    mx = fmax(mx, u);
  }
  s_min[threadIdx.x] = mn;
  s_max[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + o]);
      s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + o]);
    }
    __syncthreads();
  }
  double u0 = 0.5 * (s_min[0] + s_max[0]);
  for (int i = threadIdx.x; i < t.PM * 9; i += blockDim.x) {
    double v = t.axes[i];
    float hi = (float)v;
    t.axh[i] = hi;
    t.axl[i] = (float)(v - (double)hi);
  }
  for (int k = threadIdx.x; k < t.S; k += blockDim.x) {
    float *q = t.src32 + (size_t)k * SRC32_STRIDE;
    double d = 1.0 / t.lam[k] - u0;
    float hi = (float)d;
    q[SRC32_DH] = hi;
    q[SRC32_DL] = (float)(d - (double)hi);
    q[SRC32_W] = (float)t.w[k];
    for (int c = 0; c < 3; ++c) {
      q[SRC32_DIR + c] = t.dir[c];
      q[SRC32_E + c] = t.ep[c];
      q[SRC32_B + c] = t.bp[c];
    }
  }
  if (threadIdx.x == 0) {
    *t.panel_out = t.panel;
    t.counters[0] = 0;
    t.counters[1] = 0;
    *t.u0_out = u0;
  }
}

// Device address of the scratch array on the current device, looked up
// once per device (cudaGetSymbolAddress with that device current).
int scratch_address(int dev, void **out) {
  if (dev < 0 || dev >= kMaxDevices) return NB_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return NB_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return NB_OK;
}

}  // namespace
}  // namespace nbgb

extern "C" int nb_add_spots_noalloc(
    const nb_panel *panel, int oversample, int n_layers, double thickness_m,
    double atten_m, const double *axes_pm, int n_pm, double Na, double Nb,
    double Nc, double scale, const float *F, const int hkl_min[3],
    const int hkl_n[3], int interp, double default_F, const double *lambda_A,
    const double *weights, int n_src, const double dir[3], double fluence,
    double kahn_K, const double e_vec[3], double *image, void *cuda_stream) {
  nbgb::NvtxRange nvtx_("nb_add_spots_noalloc");
  using namespace nbgb;
  // ---- argument checks (host values only)
  if (!panel || !axes_pm || !F || !hkl_min || !hkl_n || !lambda_A ||
      !weights || !dir || !e_vec || !image)
    return NB_EINVAL;
  if (n_pm < 1 || n_pm > kNoAllocMaxPM || n_src < 1 || n_src > kNoAllocMaxSrc)
    return NB_EINVAL;  // beyond the scratch array's tables
  if (oversample < 1 || n_layers < 1 || oversample * oversample * n_layers > 32)
    return NB_EINVAL;
  if (panel->nfast < 1 || panel->nslow < 1 || !(panel->pixel_m > 0))
    return NB_EINVAL;
  if (!(thickness_m >= 0) || (thickness_m == 0 && n_layers != 1) ||
      (thickness_m > 0 && !(atten_m > 0)))
    return NB_EINVAL;
  if (!(Na > 0) || !(Nb > 0) || !(Nc > 0) || !(kahn_K >= 0 && kahn_K <= 1))
    return NB_EINVAL;
  if (interp != NB_INTERP_NEAREST && interp != NB_INTERP_TRICUBIC)
    return NB_EINVAL;
  for (int i = 0; i < 3; ++i)
    if (hkl_n[i] < 1) return NB_EINVAL;
  double dn = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  if (std::fabs(dn - 1.0) > 1e-9) return NB_EINVAL;
  double de = dir[0] * e_vec[0] + dir[1] * e_vec[1] + dir[2] * e_vec[2];
  double ep[3] = {e_vec[0] - de * dir[0], e_vec[1] - de * dir[1],
                  e_vec[2] - de * dir[2]};
  double en = std::sqrt(ep[0] * ep[0] + ep[1] * ep[1] + ep[2] * ep[2]);
  if (!(en > 0)) return NB_EINVAL;
  for (double &v : ep) v /= en;
  double bp[3] = {dir[1] * ep[2] - dir[2] * ep[1],
                  dir[2] * ep[0] - dir[0] * ep[2],
                  dir[0] * ep[1] - dir[1] * ep[0]};

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return NB_ECUDA;
  }
  void *base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc != NB_OK) return rc;
  unsigned char *sc = (unsigned char *)base;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // ---- the kernel arguments: tables and panel in the scratch array
  SpotArgs a;
  std::memset(&a, 0, sizeof a);
  DevPanel P;
  std::memset(&P, 0, sizeof P);
  for (int c = 0; c < 3; ++c) {
    P.origin[c] = panel->origin[c];
    P.fdir[c] = panel->fdir[c];
    P.sdir[c] = panel->sdir[c];
    P.ndir[c] = panel->ndir[c];
  }
  P.px = panel->pixel_m;
  P.nfast = panel->nfast;
  P.nslow = panel->nslow;
  P.pix0 = 0;
  P.tiles_f = (P.nfast + kTileF - 1) / kTileF;
  P.tiles = P.tiles_f * ((P.nslow + kTileS - 1) / kTileS);
  panel_ff(P);
  float *axh = (float *)sc;
  float *axl = axh + (size_t)n_pm * 9;
  float *src32 = axl + (size_t)n_pm * 9;
  DevPanel *dpanel = (DevPanel *)(sc + kPanelOffset);
  unsigned long long *counters = (unsigned long long *)(sc + kCounterOffset);
  double *u0_dev = (double *)(counters + 2);

  a.panels = dpanel;
  a.n_panels = 1;
  a.n_tiles = P.tiles;
  a.npix = (long long)P.nfast * P.nslow;
  a.os = oversample;
  a.T = n_layers;
  a.dt = thickness_m > 0 ? thickness_m / n_layers : 0.0;
  a.thickness = thickness_m;
  a.atten = atten_m;
  a.PM = n_pm;
  a.axh = axh;
  a.axl = axl;
  double N[3] = {Na, Nb, Nc};
  for (int i = 0; i < 3; ++i) {
    a.N64[i] = N[i];
    a.N[i] = (float)N[i];
    a.hmin[i] = hkl_min[i];
    a.hn[i] = hkl_n[i];
    a.i0[i] = dir[i];
    a.e0[i] = ep[i];
    a.b0[i] = bp[i];
  }
  double nn = Na * Nb * Nc;
  a.N6 = (float)(nn * nn);
  a.shape = NB_SHAPE_GAUSS;
  a.interp = interp;
  a.F = F;
  a.defF = (float)default_F;
  a.defF64 = default_F;
  a.S = n_src;
  a.src32 = src32;
  a.kahn = (float)kahn_K;
  a.kahn64 = kahn_K;
  a.has_div = 0;
  a.prefactor = kElectronRadius * kElectronRadius * fluence * scale /
                ((double)oversample * oversample * n_pm);
  a.image = image;
  a.stats = counters + 1;
  args_ff(a);
  if (!split_supported(a)) return NB_EINVAL;

  TableArgs t;
  std::memset(&t, 0, sizeof t);
  t.axes = axes_pm;
  t.lam = lambda_A;
  t.w = weights;
  t.PM = n_pm;
  t.S = n_src;
  for (int c = 0; c < 3; ++c) {
    t.dir[c] = (float)dir[c];
    t.ep[c] = (float)ep[c];
    t.bp[c] = (float)bp[c];
  }
  t.panel = P;
  t.axh = axh;
  t.axl = axl;
  t.src32 = src32;
  t.panel_out = dpanel;
  t.counters = counters;
  t.u0_out = u0_dev;
  noalloc_tables_kernel<<<1, 256, 0, st>>>(t);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return NB_ECUDA;
  // u0 (double-float) is a kernel argument of the spots kernel: read it
  // back into host stack memory (the table kernel computed it on device)
  double u0 = 0.0;
  e = cudaMemcpyAsync(&u0, u0_dev, sizeof u0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return NB_ECUDA;
  a.u0 = u0;
  a.u0h = (float)u0;
  a.u0l = (float)(u0 - (double)a.u0h);
  int sm_count = 0;
  if (cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev) !=
      cudaSuccess) {
    cudaGetLastError();
    return NB_ECUDA;
  }
  e = launch_spots_split(a, counters, sm_count, st);
  return e == cudaSuccess ? NB_OK : NB_ECUDA;
}
