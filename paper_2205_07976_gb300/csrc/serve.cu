// serve.cu -- continuous batching of Bragg-spot shots on one GPU.
//
// The paper hides I/O latency by letting several MPI ranks share one GPU,
// each simulating its own batch of images (Sec. IV, Fig. 3).  Here one
// server process keeps the crystal's structure-factor table and the
// detector resident and admits shot requests of uneven size (ROI pixels,
// sources, mosaic domains) as slots and device memory free up:
//
//   submit  -> FIFO queue (inputs copied, tables built on the host)
//   step    -> admit while a slot and room in the image pool exist (first
//              fit; a blocked head request stops bypassing after 8 steps);
//              cut the active requests into work items (128 pixels for the
//              thread kernel, 64 for the warp kernel) up to a pixel-step
//              budget: half shared equally by the running requests, the
//              rest to the oldest first; replay one of two CUDA graphs
//              (work list upload from its own pinned buffer, counter reset,
//              the two persistent kernels); then wait for the step queued
//              by the previous call, so the GPU runs one step while the host
//              prepares the next; requests whose last item ran in a
//              finished step are complete
//   result  -> copy the image out on a separate stream, free its pool
//              range (its slot was freed when the request completed)
//
// The persistent kernels' blocks pull work items through atomic counters;
// each item stages its request's tables in shared memory and computes its
// pixels with the same device functions as the stand-alone kernels (one
// thread per pixel, or one warp per pixel for the requests the stand-alone
// library would run that way), so a request's image does not depend on
// what it was batched with.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "../../include/nbgb.h"
#include "mixed_pixel.cuh"
#include "split_pixel.cuh"

namespace nbgb {

constexpr int kServeMaxPM = 64;
constexpr int kServeMaxSrc = 128;
constexpr int kServeItemPixels = kTileThreads;  // one pixel per thread
constexpr int kServeWarpItemPixels = 64;  // warp kernel: 16 pixels per warp
constexpr int kServeMaxItems = 16384;

struct SlotParams {
  float axh[kServeMaxPM * 9];
  float axl[kServeMaxPM * 9];
  float src32[kServeMaxSrc * SRC32_STRIDE];
  int PM, S;
  float u0h, u0l;
  double prefactor;
  int f0, s0, nf, ns;
  long long img_off;  // element offset in the image pool
};

struct WorkItem {
  int slot;
  int count;
  long long first;  // first ROI pixel (row-major in the ROI)
};

struct WorkList {
  int n;
  int pad[3];
  WorkItem items[kServeMaxItems];
};

template <int INTERP>
__global__ void __launch_bounds__(kTileThreads, 4)
    serve_kernel(SpotArgs base, const SlotParams *slots, const WorkList *wl,
                 unsigned *counter, double *pool) {
  __shared__ float s_axh[kServeMaxPM * 9];
  __shared__ float s_axl[kServeMaxPM * 9];
  __shared__ float s_src[kServeMaxSrc * SRC32_STRIDE];
  __shared__ int s_item;
  int staged = -1;
  const DevPanel &P = base.panels[0];
  const int n = wl->n;
  while (true) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    int it = s_item;
    __syncthreads();
    if (it >= n) break;
    const WorkItem w = wl->items[it];
    const SlotParams &sp = slots[w.slot];
    if (w.slot != staged) {
      for (int i = threadIdx.x; i < sp.PM * 9; i += blockDim.x) {
        s_axh[i] = sp.axh[i];
        s_axl[i] = sp.axl[i];
      }
      for (int i = threadIdx.x; i < sp.S * SRC32_STRIDE; i += blockDim.x)
        s_src[i] = sp.src32[i];
      staged = w.slot;
      __syncthreads();
    }
    if ((int)threadIdx.x < w.count) {
      long long p = w.first + threadIdx.x;
      int s = sp.s0 + (int)(p / sp.nf);
      int f = sp.f0 + (int)(p % sp.nf);
      const PixelView v{sp.PM, sp.S, sp.u0h, sp.u0l};
      unsigned evals = 0;
      double total = mixed_pixel<1, INTERP, 0, 0>(base, v, s_axh, s_axl,
                                                  s_src, P, s, f, evals);
      pool[sp.img_off + p] = sp.prefactor * total;
    }
    __syncthreads();
  }
}

// The warp-per-pixel form for requests the stand-alone library would also
// run one warp per pixel (tricubic lookup, >= 8 subpixel x mosaic items):
// each work item stages its request's tables once, then each warp sums its
// pixels with the same device function as the stand-alone kernel.
template <int INTERP>
__global__ void __launch_bounds__(kSplitThreads, 5)
    serve_warp_kernel(SpotArgs base, const SlotParams *slots,
                      const WorkList *wl, unsigned *counter, double *pool) {
  extern __shared__ float sms[];
  __shared__ int s_item;
  const DevPanel &P = base.panels[0];
  const int n = wl->n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int staged = -1;
  SplitBlock b;
  SplitCounts cnt;
  const int U = base.os * base.os * base.T;
  const int B = kMaxUnits / U;
  while (true) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    int it = s_item;
    __syncthreads();
    if (it >= n) break;
    const WorkItem w = wl->items[it];
    const SlotParams &sp = slots[w.slot];
    if (w.slot != staged) {
      split_stage(b, sms, base, sp.axh, sp.axl, sp.src32, sp.PM, sp.S, sp.u0h,
                  sp.u0l);
      staged = w.slot;
    }
    // the warp's pixels j = warp, warp + 4, ...: sub-pixel units of B of
    // them at a time in one pass (the FP64 geometry fills the lanes), then
    // the sums one after another
    float *unit = b.unit_base + warp * kMaxUnits * kUnitFloats;
    const int npx = (w.count - warp + kSplitWarps - 1) / kSplitWarps;
    for (int i0 = 0; i0 < npx; i0 += B) {
      const int nb = min(B, npx - i0);
      if (lane < nb * U) {
        const int bi = lane / U;
        const long long p = w.first + warp + (long long)(i0 + bi) * kSplitWarps;
        const int s = sp.s0 + (int)(p / sp.nf);
        const int f = sp.f0 + (int)(p % sp.nf);
        split_unit<0>(base, P, s, f, lane - bi * U, unit + lane * kUnitFloats);
      }
      __syncwarp();
      for (int bi = 0; bi < nb; ++bi) {
        const long long p = w.first + warp + (long long)(i0 + bi) * kSplitWarps;
        const double v = split_sum<INTERP, 0>(
            base, b, unit + bi * U * kUnitFloats, cnt);
        if (lane == 0) pool[sp.img_off + p] = sp.prefactor * v;
      }
      __syncwarp();  // the next batch rewrites the units
    }
    __syncthreads();  // the tables may be restaged for the next item
  }
}

size_t serve_warp_smem_bytes() {
  SpotArgs a;
  memset(&a, 0, sizeof a);
  a.PM = kServeMaxPM;
  a.S = kServeMaxSrc;
  return split_smem_bytes(a);
}

}  // namespace nbgb

using nbgb::SlotParams;
using nbgb::WorkItem;
using nbgb::WorkList;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Buf {
  void *p = nullptr;
  cudaError_t alloc(size_t n) { return cudaMalloc(&p, n); }
  ~Buf() {
    if (p) cudaFree(p);
  }
};

struct Request {
  long long id;
  SlotParams params;  // host copy (img_off set at admission)
  long long npix, steps_per_pixel;
  long long next = 0;     // next ROI pixel to schedule
  long long last_step = -1;  // the step holding its last work item
  int slot = -1;
  long long pool_off = -1;
  int state = NB_REQ_QUEUED;
  int blocked_steps = 0;
  bool warp = false;  // computed by the warp-per-pixel kernel
};

}  // namespace

struct nb_server {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sm_count = 0, blocks = 0;
  int max_slots = 0;
  long long pool_elems = 0;
  long long budget = 0;
  double timeout_s = 60.0;
  std::string err;
  // shared resident state
  nb_panel panel;
  int os = 1, T = 1;
  double thick = 0, atten = 0;
  double N[3] = {1, 1, 1};
  int shape = NB_SHAPE_GAUSS, interp = NB_INTERP_TRICUBIC;
  int hmin[3], hn[3];
  double defF = 0;
  double fluence = 0, kahn = 0, evec[3] = {1, 0, 0}, dir[3] = {0, 0, 1};
  Buf d_F, d_F4, d_C4, d_panel, d_slots, d_pool, d_work, d_work_w, d_counter;
  // two host work-list buffers, each with its graph: the next step is
  // built and queued while the previous one runs
  WorkList *h_work[2] = {nullptr, nullptr};    // pinned: thread-kernel items
  WorkList *h_work_w[2] = {nullptr, nullptr};  // pinned: warp-kernel items
  int blocks_w = 0;
  size_t smem_w = 0;
  nbgb::SpotArgs base;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaEvent_t done_ev[2] = {nullptr, nullptr};
  bool in_flight[2] = {false, false};
  long long step_of[2] = {0, 0};
  std::deque<int> flight;  // buffers in flight, oldest first
  int cur = 0;             // the buffer the next step is built in
  long long step_counter = 0;
  cudaStream_t copy_stream = nullptr;  // result copies
  // steps built in buffer b run on stream_of(b): consecutive steps overlap,
  // so the tail of one step's persistent kernels is filled by the next;
  // up_ev[b] marks the slot uploads made for a step on its stream, which
  // the next step (on the other stream) waits for
  cudaStream_t stream2 = nullptr;
  cudaEvent_t up_ev[2] = {nullptr, nullptr};
  // host bookkeeping
  long long next_id = 1;
  std::deque<long long> queue;
  std::map<long long, Request> reqs;
  std::vector<int> free_slots;
  std::map<long long, long long> free_ranges;  // offset -> length
  std::vector<long long> completed;            // not yet reported
};

static int sfail(nb_server *s, int code, const std::string &m) {
  if (s) s->err = m;
  return code;
}

// first-fit allocation in the image pool (elements)
static long long pool_alloc(nb_server *s, long long n) {
  for (auto it = s->free_ranges.begin(); it != s->free_ranges.end(); ++it) {
    if (it->second >= n) {
      long long off = it->first, len = it->second;
      s->free_ranges.erase(it);
      if (len > n) s->free_ranges[off + n] = len - n;
      return off;
    }
  }
  return -1;
}

static void pool_free(nb_server *s, long long off, long long n) {
  auto it = s->free_ranges.emplace(off, n).first;
  auto nx = std::next(it);
  if (nx != s->free_ranges.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->free_ranges.erase(nx);
  }
  if (it != s->free_ranges.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->free_ranges.erase(it);
    }
  }
}

static cudaStream_t stream_of(const nb_server *s, int b) {
  return b == 0 ? s->stream : s->stream2;
}

// The graph of one step from host buffer b, on stream_of(b): its work
// lists to its own device copies, its counters reset, the two persistent
// kernels.
static int build_graph(nb_server *s, int b) {
  cudaStream_t st = stream_of(s, b);
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return sfail(s, NB_ECUDA, "graph capture begin");
  WorkList *dw = (WorkList *)s->d_work.p + b;
  WorkList *dww = (WorkList *)s->d_work_w.p + b;
  unsigned *ctr = (unsigned *)s->d_counter.p + 2 * b;
  cudaMemcpyAsync(dw, s->h_work[b], sizeof(WorkList), cudaMemcpyHostToDevice,
                  st);
  cudaMemcpyAsync(dww, s->h_work_w[b], sizeof(WorkList),
                  cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), st);
  void (*kern)(nbgb::SpotArgs, const SlotParams *, const WorkList *,
               unsigned *, double *) =
      s->interp ? nbgb::serve_kernel<1> : nbgb::serve_kernel<0>;
  kern<<<s->blocks, nbgb::kTileThreads, 0, st>>>(
      s->base, (const SlotParams *)s->d_slots.p, dw, ctr,
      (double *)s->d_pool.p);
  if (s->interp == NB_INTERP_TRICUBIC) {
    nbgb::serve_warp_kernel<1><<<s->blocks_w, nbgb::kSplitThreads, s->smem_w,
                                 st>>>(
        s->base, (const SlotParams *)s->d_slots.p, dww, ctr + 1,
        (double *)s->d_pool.p);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(st, &g);
  if (e != cudaSuccess) return sfail(s, NB_ECUDA, "graph capture end");
  e = cudaGraphInstantiate(&s->graph[b], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return sfail(s, NB_ECUDA, "graph instantiate");
  return NB_OK;
}

extern "C" {

int nb_server_create(nb_server **out, int device, void *cuda_stream,
                     int max_slots, long long pool_bytes, long long step_budget,
                     const nb_panel *panel, int oversample, int n_layers,
                     double thickness_m, double atten_m, const float *F,
                     const int hkl_min[3], const int hkl_n[3], int interp,
                     double default_F, double Na, double Nb, double Nc,
                     const double dir[3], double fluence, double kahn_K,
                     const double e_vec[3]) {
  nbgb::NvtxRange nvtx_("nb_server_create");
  if (!out) return NB_EINVAL;
  *out = nullptr;
  if (!panel || !F || !hkl_min || !hkl_n || !dir || !e_vec) return NB_EINVAL;
  if (max_slots < 1 || max_slots > 4096 || pool_bytes < 8) return NB_EINVAL;
  if (oversample < 1 || n_layers < 1 || oversample > 8 || n_layers > 8)
    return NB_EINVAL;
  if (!(thickness_m >= 0) || (thickness_m == 0 && n_layers != 1) ||
      (thickness_m > 0 && !(atten_m > 0)))
    return NB_EINVAL;
  if (panel->nfast < 1 || panel->nslow < 1 || !(panel->pixel_m > 0))
    return NB_EINVAL;
  if (interp != NB_INTERP_NEAREST && interp != NB_INTERP_TRICUBIC)
    return NB_EINVAL;
  if (!(Na > 0 && Nb > 0 && Nc > 0) || !(kahn_K >= 0 && kahn_K <= 1))
    return NB_EINVAL;
  for (int i = 0; i < 3; ++i)
    if (hkl_n[i] < 1) return NB_EINVAL;
  double dn = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  if (std::fabs(dn - 1.0) > 1e-9) return NB_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 ||
      device >= ndev) {
    cudaGetLastError();
    return NB_ECUDA;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  nb_server *s = new (std::nothrow) nb_server();
  if (!s) return NB_ENOMEM;
  int rc = NB_OK;
  do {
    s->device = device;
    s->max_slots = max_slots;
    s->pool_elems = pool_bytes / (long long)sizeof(double);
    s->budget = step_budget > 0 ? step_budget : 1000000000LL;
    s->panel = *panel;
    s->os = oversample;
    s->T = n_layers;
    s->thick = thickness_m;
    s->atten = atten_m;
    s->N[0] = Na;
    s->N[1] = Nb;
    s->N[2] = Nc;
    s->interp = interp;
    s->defF = default_F;
    s->fluence = fluence;
    s->kahn = kahn_K;
    std::memcpy(s->evec, e_vec, sizeof s->evec);
    std::memcpy(s->dir, dir, sizeof s->dir);
    for (int i = 0; i < 3; ++i) {
      s->hmin[i] = hkl_min[i];
      s->hn[i] = hkl_n[i];
    }
    if (cuda_stream) {
      s->stream = (cudaStream_t)cuda_stream;
    } else {
      if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) !=
          cudaSuccess) {
        rc = sfail(s, NB_ECUDA, "stream");
        break;
      }
      s->own_stream = true;
    }
    if (cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount,
                               device) != cudaSuccess) {
      rc = NB_ECUDA;
      break;
    }
    size_t nF = (size_t)hkl_n[0] * hkl_n[1] * hkl_n[2];
    if (s->d_F.alloc(nF * 4) != cudaSuccess ||
        s->d_panel.alloc(sizeof(nbgb::DevPanel)) != cudaSuccess ||
        s->d_slots.alloc(sizeof(SlotParams) * (size_t)max_slots) !=
            cudaSuccess ||
        s->d_pool.alloc((size_t)s->pool_elems * sizeof(double)) !=
            cudaSuccess ||
        s->d_work.alloc(2 * sizeof(WorkList)) != cudaSuccess ||
        s->d_work_w.alloc(2 * sizeof(WorkList)) != cudaSuccess ||
        s->d_counter.alloc(4 * sizeof(unsigned)) != cudaSuccess ||
        cudaHostAlloc((void **)&s->h_work[0], sizeof(WorkList),
                      cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&s->h_work_w[0], sizeof(WorkList),
                      cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&s->h_work[1], sizeof(WorkList),
                      cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&s->h_work_w[1], sizeof(WorkList),
                      cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      rc = sfail(s, NB_ENOMEM, "server buffers");
      break;
    }
    for (int b = 0; b < 2; ++b) {
      std::memset(s->h_work[b], 0, sizeof(WorkList));
      std::memset(s->h_work_w[b], 0, sizeof(WorkList));
    }
    cudaMemcpy(s->d_F.p, F, nF * 4, cudaMemcpyHostToDevice);
    nbgb::DevPanel P;
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
    nbgb::panel_ff(P);
    cudaMemcpy(s->d_panel.p, &P, sizeof P, cudaMemcpyHostToDevice);
    // shared kernel arguments
    nbgb::SpotArgs &a = s->base;
    std::memset(&a, 0, sizeof a);
    a.panels = (const nbgb::DevPanel *)s->d_panel.p;
    a.n_panels = 1;
    a.os = oversample;
    a.T = n_layers;
    a.dt = thickness_m > 0 ? thickness_m / n_layers : 0.0;
    a.thickness = thickness_m;
    a.atten = atten_m;
    double ep[3], bp[3];
    {
      double de = dir[0] * e_vec[0] + dir[1] * e_vec[1] + dir[2] * e_vec[2];
      for (int c = 0; c < 3; ++c) ep[c] = e_vec[c] - de * dir[c];
      double en = std::sqrt(ep[0] * ep[0] + ep[1] * ep[1] + ep[2] * ep[2]);
      if (!(en > 0)) {
        rc = sfail(s, NB_EINVAL, "e_vec parallel to the beam");
        break;
      }
      for (double &v : ep) v /= en;
      bp[0] = dir[1] * ep[2] - dir[2] * ep[1];
      bp[1] = dir[2] * ep[0] - dir[0] * ep[2];
      bp[2] = dir[0] * ep[1] - dir[1] * ep[0];
    }
    for (int i = 0; i < 3; ++i) {
      a.N64[i] = s->N[i];
      a.N[i] = (float)s->N[i];
      a.hmin[i] = hkl_min[i];
      a.hn[i] = hkl_n[i];
      a.i0[i] = dir[i];
      a.e0[i] = ep[i];
      a.b0[i] = bp[i];
    }
    nbgb::args_ff(a);
    double nn = Na * Nb * Nc;
    a.N6 = (float)(nn * nn);
    a.shape = NB_SHAPE_GAUSS;
    a.interp = interp;
    a.F = (const float *)s->d_F.p;
    if (interp == NB_INTERP_TRICUBIC && s->d_F4.alloc(nF * sizeof(float4)) ==
                                            cudaSuccess &&
        nbgb::build_sliding_table((const float *)s->d_F.p, s->hn,
                                  (float4 *)s->d_F4.p, s->stream) ==
            cudaSuccess) {
      cudaStreamSynchronize(s->stream);
      a.F4 = (const float4 *)s->d_F4.p;
    }
    cudaGetLastError();
    // the tricubic polynomial of every cell, as the stand-alone warp
    // kernel uses it (same results bit for bit)
    // (not for an axis longer than 1000 nodes: the warp kernel packs a
    // table index into 10 bits per axis)
    if (interp == NB_INTERP_TRICUBIC && hkl_n[0] >= 4 && hkl_n[1] >= 4 &&
        hkl_n[2] >= 4 && hkl_n[0] <= 1000 && hkl_n[1] <= 1000 &&
        hkl_n[2] <= 1000) {
      size_t cells =
          (size_t)(hkl_n[0] - 3) * (hkl_n[1] - 3) * (hkl_n[2] - 3);
      if (cells * 16 * sizeof(float4) <= ((size_t)2 << 30) &&
          s->d_C4.alloc(cells * 16 * sizeof(float4)) == cudaSuccess &&
          nbgb::build_cell_polynomials((const float *)s->d_F.p, s->hn,
                                       (float4 *)s->d_C4.p,
                                       s->stream) == cudaSuccess) {
        cudaStreamSynchronize(s->stream);
        a.C4 = (const float4 *)s->d_C4.p;
      }
      cudaGetLastError();
    }
    a.defF = (float)default_F;
    a.defF64 = default_F;
    a.kahn = (float)kahn_K;
    a.kahn64 = kahn_K;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, interp ? nbgb::serve_kernel<1> : nbgb::serve_kernel<0>,
        nbgb::kTileThreads, 0);
    s->blocks = s->sm_count * (per_sm > 0 ? per_sm : 1);
    if (interp == NB_INTERP_TRICUBIC) {
      s->smem_w = nbgb::serve_warp_smem_bytes();
      cudaFuncSetAttribute(nbgb::serve_warp_kernel<1>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)s->smem_w);
      int per_sm_w = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm_w, nbgb::serve_warp_kernel<1>, nbgb::kSplitThreads,
          s->smem_w);
      s->blocks_w = s->sm_count * (per_sm_w > 0 ? per_sm_w : 1);
    }
    for (int i = max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->free_ranges[0] = s->pool_elems;
    if (cudaEventCreateWithFlags(&s->done_ev[0], cudaEventDisableTiming) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&s->done_ev[1], cudaEventDisableTiming) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stream2, cudaStreamNonBlocking) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&s->up_ev[0], cudaEventDisableTiming) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&s->up_ev[1], cudaEventDisableTiming) !=
            cudaSuccess) {
      rc = NB_ECUDA;
      break;
    }
    rc = build_graph(s, 0);
    if (rc == NB_OK) rc = build_graph(s, 1);
  } while (false);
  if (cudaGetLastError() != cudaSuccess && rc == NB_OK) rc = NB_ECUDA;
  cudaSetDevice(prev);
  if (rc != NB_OK) {
    nb_server_free(s);
    return rc;
  }
  *out = s;
  return NB_OK;
}

int nb_server_free(nb_server *s) {
  if (!s) return NB_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->stream2) {
    cudaStreamSynchronize(s->stream2);
    cudaStreamDestroy(s->stream2);
  }
  if (s->copy_stream) {
    cudaStreamSynchronize(s->copy_stream);
    cudaStreamDestroy(s->copy_stream);
  }
  for (int b = 0; b < 2; ++b) {
    if (s->graph[b]) cudaGraphExecDestroy(s->graph[b]);
    if (s->done_ev[b]) cudaEventDestroy(s->done_ev[b]);
    if (s->up_ev[b]) cudaEventDestroy(s->up_ev[b]);
    if (s->h_work[b]) cudaFreeHost(s->h_work[b]);
    if (s->h_work_w[b]) cudaFreeHost(s->h_work_w[b]);
  }
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  {
    Buf *bufs[] = {&s->d_F,    &s->d_F4,     &s->d_C4,     &s->d_panel,
                   &s->d_slots, &s->d_pool, &s->d_work, &s->d_work_w,
                   &s->d_counter};
    for (Buf *b : bufs) {
      if (b->p) cudaFree(b->p);
      b->p = nullptr;
    }
  }
  delete s;
  cudaSetDevice(prev);
  return NB_OK;
}

const char *nb_server_last_error(const nb_server *s) {
  return s ? s->err.c_str() : "null server";
}

int nb_server_submit(nb_server *s, const double axes[9], const double *umats,
                     int n_mosaic, const double *lambda_A,
                     const double *weights, int n_src, double scale,
                     int roi_f0, int roi_s0, int roi_nf, int roi_ns,
                     long long *request_id) {
  nbgb::NvtxRange nvtx_("nb_server_submit");
  if (!s) return NB_EINVAL;
  if (!axes || !umats || !lambda_A || !weights || !request_id)
    return sfail(s, NB_EINVAL, "NULL argument");
  if (n_mosaic < 1 || n_mosaic > nbgb::kServeMaxPM || n_src < 1 ||
      n_src > nbgb::kServeMaxSrc)
    return sfail(s, NB_EINVAL, "need 1 <= n_mosaic <= 64, 1 <= n_src <= 128");
  if (roi_nf < 1 || roi_ns < 1 || roi_f0 < 0 || roi_s0 < 0 ||
      roi_f0 + roi_nf > s->panel.nfast || roi_s0 + roi_ns > s->panel.nslow)
    return sfail(s, NB_EINVAL, "ROI outside the detector");
  long long npix = (long long)roi_nf * roi_ns;
  if (npix > s->pool_elems)
    return sfail(s, NB_EINVAL, "ROI larger than the whole image pool");
  for (int k = 0; k < n_src; ++k)
    if (!(lambda_A[k] > 0)) return sfail(s, NB_EINVAL, "wavelength");
  Request r;
  r.id = s->next_id++;
  std::memset(&r.params, 0, sizeof r.params);
  std::vector<double> ax;
  double spindle[3] = {0, 1, 0};
  nbgb::rotated_axes_table(axes, umats, n_mosaic, 1, 0.0, 0.0, spindle, ax);
  std::vector<double> dirs(3 * (size_t)n_src);
  for (int k = 0; k < n_src; ++k)
    for (int c = 0; c < 3; ++c) dirs[3 * k + c] = s->dir[c];
  std::vector<double> lam(lambda_A, lambda_A + n_src),
      wts(weights, weights + n_src);
  nbgb::sort_sources(dirs, lam, wts);  // the order nb_set_beam uses
  double u0 = nbgb::source_u0(lam.data(), n_src);
  std::vector<float> axh, axl, src32;
  nbgb::shot_tables_f32(ax, lam.data(), wts.data(), dirs.data(), n_src,
                        s->evec, u0, false, axh, axl, src32);
  std::memcpy(r.params.axh, axh.data(), axh.size() * 4);
  std::memcpy(r.params.axl, axl.data(), axl.size() * 4);
  std::memcpy(r.params.src32, src32.data(), src32.size() * 4);
  r.params.PM = n_mosaic;
  r.params.S = n_src;
  r.params.u0h = (float)u0;
  r.params.u0l = (float)(u0 - (double)r.params.u0h);
  r.params.prefactor = nbgb::kElectronRadius * nbgb::kElectronRadius *
                       s->fluence * scale /
                       ((double)s->os * s->os * n_mosaic);
  r.params.f0 = roi_f0;
  r.params.s0 = roi_s0;
  r.params.nf = roi_nf;
  r.params.ns = roi_ns;
  r.npix = npix;
  r.steps_per_pixel =
      (long long)s->os * s->os * s->T * n_src * (long long)n_mosaic;
  // the same choice as nb_add_spots makes for this shot
  r.warp = s->interp == NB_INTERP_TRICUBIC &&
           (long long)s->os * s->os * s->T * n_mosaic >= 8 &&
           s->os * s->os * s->T <= 32;
  s->queue.push_back(r.id);
  *request_id = r.id;
  s->reqs.emplace(r.id, std::move(r));
  return NB_OK;
}

// admission: FIFO; later requests may pass a head that does not fit until
// the head has waited 8 steps
static int admit(nb_server *s) {
  bool head_blocked_long = false;
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    if (s->free_slots.empty()) break;
    Request &r = s->reqs[*it];
    long long off = pool_alloc(s, r.npix);
    if (off < 0) {
      if (it == s->queue.begin() && ++r.blocked_steps > 8)
        head_blocked_long = true;
      if (head_blocked_long) break;
      ++it;
      continue;
    }
    r.slot = s->free_slots.back();
    s->free_slots.pop_back();
    r.pool_off = off;
    r.params.img_off = off;
    r.state = NB_REQ_RUNNING;
    cudaError_t e = cudaMemcpyAsync((SlotParams *)s->d_slots.p + r.slot,
                                    &r.params, sizeof(SlotParams),
                                    cudaMemcpyHostToDevice,
                                    stream_of(s, s->cur));
    if (e != cudaSuccess) return sfail(s, NB_ECUDA, "slot upload");
    it = s->queue.erase(it);
  }
  return NB_OK;
}

// Waits (up to timeout_s) for the oldest step in flight and completes the
// requests whose last work item it held: their slots are free again; their
// images stay in the pool until nb_server_result fetches them.
static int finish_oldest(nb_server *s, double timeout_s) {
  if (s->flight.empty()) return NB_OK;
  const int b = s->flight.front();
  double t0 = now_s();
  while (true) {
    cudaError_t q = cudaEventQuery(s->done_ev[b]);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return sfail(s, NB_ECUDA, "step failed");
    if (now_s() - t0 > timeout_s)
      return sfail(s, NB_ETIMEOUT, "step did not finish in time");
  }
  s->flight.pop_front();
  s->in_flight[b] = false;
  for (auto &kv : s->reqs) {
    Request &r = kv.second;
    if (r.state != NB_REQ_RUNNING || r.next < r.npix ||
        r.last_step != s->step_of[b])
      continue;
    r.state = NB_REQ_DONE;
    s->free_slots.push_back(r.slot);
    r.slot = -1;
    s->completed.push_back(r.id);
  }
  return NB_OK;
}

static bool any_schedulable(const nb_server *s) {
  for (auto &kv : s->reqs)
    if (kv.second.state == NB_REQ_RUNNING && kv.second.next < kv.second.npix)
      return true;
  return false;
}

int nb_server_step(nb_server *s, double timeout_s, int *n_active) {
  nbgb::NvtxRange nvtx_("nb_server_step");
  if (!s) return NB_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  int rc = NB_OK;
  // the buffer this step is built in must be free (it is, unless an earlier
  // step returned on a timeout with two steps in flight)
  if (s->in_flight[s->cur]) rc = finish_oldest(s, timeout_s);
  if (rc == NB_OK) rc = admit(s);
  if (rc == NB_OK) {
    std::vector<Request *> act, finished;
    std::vector<long long> next0;  // to undo the cut if the launch fails
    for (auto &kv : s->reqs)
      if (kv.second.state == NB_REQ_RUNNING && kv.second.next < kv.second.npix) {
        act.push_back(&kv.second);
        next0.push_back(kv.second.next);
      }
    WorkList *wl = s->h_work[s->cur], *ww = s->h_work_w[s->cur];
    int nt = 0, nw = 0;
    long long used = 0;
    // half of the budget is shared equally by the active requests (at
    // least one work item each, so none starves and a new request is not
    // stuck behind an old large one), the rest goes to the oldest requests
    // first: fewer requests per step means fewer table restagings per
    // block, and requests finish sooner (act is in arrival order: the map
    // is keyed by request id)
    const long long share =
        act.empty() ? 0 : s->budget / (2 * (long long)act.size());
    for (int pass = 0; pass < 2 && used < s->budget; ++pass) {
      for (size_t j = 0; j < act.size() && used < s->budget; ++j) {
        Request &r = *act[j];
        WorkList *L = r.warp ? ww : wl;
        int &n = r.warp ? nw : nt;
        const long long cap = r.warp ? nbgb::kServeWarpItemPixels
                                     : nbgb::kServeItemPixels;
        long long mine = 0;  // pixel-steps given to r in this pass
        for (int k = 0; r.next < r.npix && used < s->budget &&
                        n < nbgb::kServeMaxItems &&
                        (pass == 1 || k < 1 || mine < share);
             ++k) {
          long long cnt = r.npix - r.next;
          if (cnt > cap) cnt = cap;
          L->items[n].slot = r.slot;
          L->items[n].count = (int)cnt;
          L->items[n].first = r.next;
          ++n;
          r.next += cnt;
          if (r.next >= r.npix) finished.push_back(&r);
          used += cnt * r.steps_per_pixel;
          mine += cnt * r.steps_per_pixel;
        }
      }
    }
    wl->n = nt;
    ww->n = nw;
    if (nt + nw > 0) {
      const int b = s->cur;
      cudaStream_t st = stream_of(s, b);
      // this step's slot uploads are on st; those of the previous build
      // are on the other stream: wait for them (not for its kernels)
      cudaError_t e = cudaEventRecord(s->up_ev[b], st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->up_ev[b ^ 1], 0);
      if (e == cudaSuccess) e = cudaGraphLaunch(s->graph[b], st);
      if (e == cudaSuccess) e = cudaEventRecord(s->done_ev[b], st);
      if (e != cudaSuccess) {
        for (size_t j = 0; j < act.size(); ++j) act[j]->next = next0[j];
        rc = sfail(s, NB_ECUDA, "graph launch");
      } else {
        s->in_flight[b] = true;
        s->step_of[b] = ++s->step_counter;
        for (Request *r : finished) r->last_step = s->step_of[b];
        s->flight.push_back(b);
        s->cur ^= 1;
        // keep one step queued behind the running one
        if (s->flight.size() > 1) rc = finish_oldest(s, timeout_s);
      }
    } else {
      // nothing new to run: drain the steps in flight
      const size_t done_before = s->completed.size();
      while (rc == NB_OK && !s->flight.empty()) rc = finish_oldest(s, timeout_s);
      // a stall only when this call completed nothing the caller could fetch
      if (rc == NB_OK && !s->queue.empty() &&
          s->completed.size() == done_before) {
        const size_t before = s->queue.size();
        rc = admit(s);
        if (rc == NB_OK && s->queue.size() == before && !any_schedulable(s))
          // nothing runs and nothing can be admitted: the pool is held by
          // completed images that were not fetched yet
          rc = sfail(s, NB_ESTATE,
                     "queued requests cannot be admitted: fetch completed "
                     "results (nb_server_result) to free the image pool");
      }
    }
  }
  if (n_active) {
    int na = 0;
    for (auto &kv : s->reqs)
      if (kv.second.state == NB_REQ_RUNNING) ++na;
    *n_active = na + (int)s->queue.size();
  }
  cudaSetDevice(prev);
  return rc;
}

int nb_server_completed(nb_server *s, long long *ids, int max_ids,
                        int *n_out) {
  if (!s || !n_out || (max_ids > 0 && !ids)) return NB_EINVAL;
  int n = 0;
  while (n < max_ids && !s->completed.empty()) {
    ids[n++] = s->completed.front();
    s->completed.erase(s->completed.begin());
  }
  *n_out = n;
  return NB_OK;
}

int nb_server_state(nb_server *s, long long id, int *state) {
  if (!s || !state) return NB_EINVAL;
  auto it = s->reqs.find(id);
  *state = it == s->reqs.end() ? NB_REQ_UNKNOWN : it->second.state;
  return NB_OK;
}

int nb_server_result(nb_server *s, long long id, void *dst, size_t n_elems,
                     int dtype, int on_device) {
  nbgb::NvtxRange nvtx_("nb_server_result");
  if (!s || !dst) return NB_EINVAL;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(s, NB_EINVAL, "unknown request");
  Request &r = it->second;
  if (r.state != NB_REQ_DONE) return sfail(s, NB_ESTATE, "request not done");
  if ((long long)n_elems != r.npix)
    return sfail(s, NB_EINVAL, "n_elems differs from the ROI pixel count");
  if (dtype != NB_DTYPE_F64)
    return sfail(s, NB_EINVAL, "results are returned as float64");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  // on the copy stream: the image is complete (its last step finished), and
  // a step queued behind it on the server's stream need not be waited for
  cudaError_t e = cudaMemcpyAsync(
      dst, (double *)s->d_pool.p + r.pool_off, n_elems * sizeof(double),
      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
      s->copy_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return sfail(s, NB_ECUDA, "result copy");
  pool_free(s, r.pool_off, r.npix);
  // a fetched request is no longer reported as completed
  for (auto c = s->completed.begin(); c != s->completed.end(); ++c)
    if (*c == id) {
      s->completed.erase(c);
      break;
    }
  s->reqs.erase(it);
  return NB_OK;
}

int nb_server_info(const nb_server *s, long long *queued, long long *running,
                   long long *done, long long *pool_free_bytes) {
  if (!s) return NB_EINVAL;
  long long q = (long long)s->queue.size(), ru = 0, d = 0, fr = 0;
  for (auto &kv : s->reqs) {
    if (kv.second.state == NB_REQ_RUNNING) ++ru;
    if (kv.second.state == NB_REQ_DONE) ++d;
  }
  for (auto &kv : s->free_ranges) fr += kv.second;
  if (queued) *queued = q;
  if (running) *running = ru;
  if (done) *done = d;
  if (pool_free_bytes) *pool_free_bytes = fr * (long long)sizeof(double);
  return NB_OK;
}

}  // extern "C"
