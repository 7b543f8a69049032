// spots_mixed.cu -- FP32-bulk forms of the per-pixel Bragg-spot sum
// (nanoBraggSpots, Sec. III-B) with the fused double accumulate of addArray
// (Listing 1).
//
// NB_MIXED keeps FP64-class accuracy only where the result needs it:
//   * pixel position and direction d per subpixel/layer in FP64;
//   * G_pm = A_pm . (d - i0) and r_pm = u0 G_pm - n0 per (subpixel, phi x
//     mosaic) in double-float (~48-bit) arithmetic;
//   * per source k the fractional offset f = G delta_k + r - rint(.) in
//     double-float, delta_k = 1/lambda_k - u0, so that h - rint(h) keeps
//     ~1e-12 absolute accuracy at |h| ~ 100 (the sinc at N = 200 needs it);
//   * the lattice factor, lookup and per-step products in FP32, summed with
//     Kahan compensation per subpixel/layer, the subpixel sums in FP64.
// NB_F32 is the naive port: geometry and h = A . S in plain FP32.
//
// One thread per pixel ("direct" variant); pixels are mapped in 16x8 tiles
// so that a warp covers a 16x2 patch (neighbours share F_cell entries in
// L1).  The rotated axes and the source table live in shared memory.
#include "mixed_pixel.cuh"

namespace nbgb {

// MODE 0: NB_MIXED, MODE 1: NB_F32.  Launch bounds: 4 blocks per SM, and
// 3 for the NB_MIXED sinc with nearest lookup, whose fast path then gets
// 112 registers instead of 104 (still 4 blocks per SM by registers) and
// measured 6.98 -> 6.91 ms on the 1024^2 sweep; the tricubic forms would
// exceed 128 registers and lose a block per SM
template <int SHAPE, int INTERP, int MODE, int HASDIV>
__global__ void __launch_bounds__(
    kTileThreads, (SHAPE == 0 && INTERP == 0 && MODE == 0) ? 3 : 4)
    spots_mixed_kernel(SpotArgs a) {
  extern __shared__ __align__(16) float smf[];
  // the sinc fast path's table (two float4 per pair of sources) first,
  // 16-byte aligned; then the axes and the source rows
  const bool fastq = SHAPE == 0 && MODE == 0 && !HASDIV && a.srcq;
  float *s_srcq = fastq ? smf : nullptr;
  const int nq = fastq ? 8 * ((a.S + 1) / 2) : 0;
  float *s_axh = smf + nq;
  float *s_axl = s_axh + a.PM * 9;
  float *s_src = s_axh + 2 * a.PM * 9;
  for (int i = threadIdx.x; i < a.PM * 9; i += blockDim.x) {
    s_axh[i] = a.axh[i];
    s_axl[i] = a.axl[i];
  }
  for (int i = threadIdx.x; i < a.S * SRC32_STRIDE; i += blockDim.x)
    s_src[i] = a.src32[i];
  if (fastq)
    for (int i = threadIdx.x; i < nq; i += blockDim.x)
      s_srcq[i] = a.srcq[i];
  __syncthreads();

  long long item = a.pixlist ? (long long)blockIdx.x * blockDim.x + threadIdx.x
                             : (long long)blockIdx.x;
  long long gp;
  int q, s, f;
  if (!map_pixel(a, item, threadIdx.x, gp, q, s, f)) return;
  const DevPanel &P = a.panels[q];
  const PixelView v{a.PM, a.S, a.u0h, a.u0l};
  unsigned evals = 0;  // terms evaluated (not skipped by the underflow cut)
  double total = mixed_pixel<SHAPE, INTERP, MODE, HASDIV>(
      a, v, s_axh, s_axl, s_src, P, s, f, evals, s_srcq);
  a.image[nb_idx(a.check, NB_SITE_IMAGE, gp, a.npix)] += a.prefactor * total;
  if (a.stats) warp_count(a.stats, evals);
}

template <int SHAPE, int INTERP, int MODE>
static void (*pick_div(int has_div))(SpotArgs) {
  return has_div ? spots_mixed_kernel<SHAPE, INTERP, MODE, 1>
                 : spots_mixed_kernel<SHAPE, INTERP, MODE, 0>;
}

template <int MODE>
static void (*pick_mode(const SpotArgs &a))(SpotArgs) {
  int key = a.shape * 2 + a.interp;
  switch (key) {
    case 0: return pick_div<0, 0, MODE>(a.has_div);
    case 1: return pick_div<0, 1, MODE>(a.has_div);
    case 2: return pick_div<1, 0, MODE>(a.has_div);
    default: return pick_div<1, 1, MODE>(a.has_div);
  }
}

__global__ void sliding_table_kernel(const float *F, int nl, long long n,
                                     float4 *F4) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int l = (int)(i % nl);
    float4 v;
    v.x = F[i];
    v.y = l + 1 < nl ? F[i + 1] : 0.f;
    v.z = l + 2 < nl ? F[i + 2] : 0.f;
    v.w = l + 3 < nl ? F[i + 3] : 0.f;
    F4[i] = v;
  }
}

cudaError_t build_sliding_table(const float *F, const int hn[3], float4 *F4,
                                cudaStream_t st) {
  long long n = (long long)hn[0] * hn[1] * hn[2];
  if (n <= 0) return cudaSuccess;
  sliding_table_kernel<<<1216, 256, 0, st>>>(F, hn[2], n, F4);
  return cudaGetLastError();
}

// monomial coefficients of the 4-point Lagrange basis on nodes -1, 0, 1, 2
// (row: node, column: power of x), exact in binary except the thirds and
// sixths
__constant__ float kLagrangeMono[4][4] = {{0.f, -1.f / 3.f, 0.5f, -1.f / 6.f},
                                          {1.f, -0.5f, -1.f, 0.5f},
                                          {0.f, 1.f, 0.5f, -0.5f},
                                          {0.f, -1.f / 6.f, 0.f, 1.f / 6.f}};

__global__ void cell_polynomials_kernel(const float *F, int nh, int nk,
                                        int nl, float4 *C4) {
  const int ch = nh - 3, ck = nk - 3, cl = nl - 3;
  const long long ncell = (long long)ch * ck * cl;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
       c < ncell; c += (long long)gridDim.x * blockDim.x) {
    int i = (int)(c / ((long long)ck * cl));
    int j = (int)((c / cl) % ck);
    int k = (int)(c % cl);
    float T[4][4][4];  // stencil, then transformed axis by axis
    for (int p = 0; p < 4; ++p)
      for (int q = 0; q < 4; ++q)
        for (int r = 0; r < 4; ++r)
          T[p][q][r] = F[((long long)(i + p) * nk + (j + q)) * nl + (k + r)];
    float U[4][4][4];
    for (int a = 0; a < 4; ++a)  // along h
      for (int q = 0; q < 4; ++q)
        for (int r = 0; r < 4; ++r) {
          float v = 0.f;
          for (int p = 0; p < 4; ++p) v = fmaf(kLagrangeMono[p][a], T[p][q][r], v);
          U[a][q][r] = v;
        }
    for (int a = 0; a < 4; ++a)  // along k
      for (int b = 0; b < 4; ++b)
        for (int r = 0; r < 4; ++r) {
          float v = 0.f;
          for (int q = 0; q < 4; ++q) v = fmaf(kLagrangeMono[q][b], U[a][q][r], v);
          T[a][b][r] = v;
        }
    float Cm[4][4][4];  // coefficient of x^a y^b z^c
    for (int a = 0; a < 4; ++a)  // along l
      for (int b = 0; b < 4; ++b)
        for (int cc = 0; cc < 4; ++cc) {
          float t = 0.f;
          for (int r = 0; r < 4; ++r) t = fmaf(kLagrangeMono[r][cc], T[a][b][r], t);
          Cm[a][b][cc] = t;
        }
    // chunks 2 (2 P + b) and 2 (2 P + b) + 1 pair the powers x^(2P) and
    // x^(2P+1) so that packed two-lane FMAs run two Horner chains in z
    float4 *out = C4 + c * 16;
    for (int P = 0; P < 2; ++P)
      for (int b = 0; b < 4; ++b) {
        const int a0 = 2 * P, a1 = 2 * P + 1;
        out[(P * 4 + b) * 2] = make_float4(Cm[a0][b][3], Cm[a1][b][3],
                                           Cm[a0][b][2], Cm[a1][b][2]);
        out[(P * 4 + b) * 2 + 1] = make_float4(Cm[a0][b][1], Cm[a1][b][1],
                                               Cm[a0][b][0], Cm[a1][b][0]);
      }
  }
}

cudaError_t build_cell_polynomials(const float *F, const int hn[3], float4 *C4,
                                   cudaStream_t st) {
  if (hn[0] < 4 || hn[1] < 4 || hn[2] < 4) return cudaErrorInvalidValue;
  cell_polynomials_kernel<<<2432, 128, 0, st>>>(F, hn[0], hn[1], hn[2], C4);
  return cudaGetLastError();
}

cudaError_t launch_spots_mixed(const SpotArgs &a, int precision,
                               cudaStream_t st) {
  // the sinc fast path's table (NB_MIXED, sinc, one beam direction)
  const bool fastq =
      a.srcq && a.shape == 0 && precision != 2 && !a.has_div;
  size_t smem = (size_t)(2 * a.PM * 9 + a.S * SRC32_STRIDE +
                         (fastq ? 8 * ((a.S + 1) / 2) : 0)) *
                sizeof(float);
  long long blocks = a.pixlist ? (a.n_list + kTileThreads - 1) / kTileThreads
                               : a.n_tiles;
  if (blocks <= 0) return cudaSuccess;
  void (*kern)(SpotArgs) =
      precision == 2 ? pick_mode<1>(a) : pick_mode<0>(a);
  cudaError_t e = cudaFuncSetAttribute(
      kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)blocks, kTileThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace nbgb
