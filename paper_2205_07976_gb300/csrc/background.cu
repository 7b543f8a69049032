// background.cu -- diffuse scatter from the air and water around the crystal
// (the addBackground kernel of Sec. IV), accumulated into the same FP64
// image as the Bragg spots.  The paper names the kernel but not its
// physics; the convention:
//
//   I_p += r_e^2 fluence n_mol / os^2 *
//          sum over subpixel, layer, source k of F_bg(stol_k)^2 w_k cap pol omega
//   stol_k = |d - i_k| / (2 lambda_k),  F_bg linear between the knots of a
//   (stol, F) table and held at its end values.
//
// One thread per pixel on the spot kernels' 16x8 pixel tiles.  The sources
// arrive grouped by direction, each group sorted by ascending 1/lambda, so
// per (subpixel, layer, group) the scattering vector |d - i|, the
// polarization and the knot search are done once: stol grows with 1/lambda,
// and the knot bracket of each further source is found by walking forward
// from the previous one.  Geometry is FP64 in both forms; the per-source
// work is FP64 (F64 form) or FP32 with a compensated sum (mixed form).
#include "nbgb_internal.cuh"

namespace nbgb {

__device__ __forceinline__ double bg_dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// bracket j with st[j] <= x < st[j + 1], for st[0] < x < st[n - 1]
template <typename T>
__device__ __forceinline__ int bg_search(const T *st, int stride, int n,
                                         T x) {
  int lo = 0, hi = n - 1;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (st[mid * stride] <= x)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

template <int F64>
__global__ void __launch_bounds__(kTileThreads)
    background_kernel(BgArgs b) {
  const SpotArgs &a = b.geo;
  extern __shared__ double smd[];
  double *s_grp = smd;                         // [G][9] dir, E', B'
  double *s_k64 = s_grp + b.n_groups * 9;      // [n][2] stol, F  (F64)
  double *s_src64 = s_k64 + (F64 ? 2 * b.n_knots : 0);  // [S][2] u, w
  float *s_k32 = (float *)(s_src64 + (F64 ? 2 * a.S : 0));  // [n][3]
  float *s_src32 = s_k32 + (F64 ? 0 : 3 * b.n_knots);       // [S][2]
  int *s_rng = (int *)(s_src32 + (F64 ? 0 : 2 * a.S));      // [G][2]
  for (int i = threadIdx.x; i < b.n_groups * 9; i += blockDim.x)
    s_grp[i] = b.grp64[i];
  for (int i = threadIdx.x; i < 2 * b.n_groups; i += blockDim.x)
    s_rng[i] = b.grp_range[i];
  if (F64) {
    for (int i = threadIdx.x; i < 2 * b.n_knots; i += blockDim.x)
      s_k64[i] = b.knots64[i];
    for (int i = threadIdx.x; i < 2 * a.S; i += blockDim.x)
      s_src64[i] = b.src64[i];
  } else {
    for (int i = threadIdx.x; i < 3 * b.n_knots; i += blockDim.x)
      s_k32[i] = b.knots32[i];
    for (int i = threadIdx.x; i < 2 * a.S; i += blockDim.x)
      s_src32[i] = b.src32[i];
  }
  __syncthreads();

  long long gp;
  int q, s, f;
  if (!map_pixel(a, (long long)blockIdx.x, threadIdx.x, gp, q, s, f)) return;
  const DevPanel &P = a.panels[q];
  const double px = P.px;
  const int os = a.os, n = b.n_knots;
  double acc = 0.0;
  for (int i = 0; i < os; ++i)
    for (int j = 0; j < os; ++j)
      for (int t = 0; t < a.T; ++t) {
        double cf = (f + (i + 0.5) / os) * px, cs = (s + (j + 0.5) / os) * px,
               cn = t * a.dt;
        double pos[3], d[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          pos[c] = P.origin[c] + cf * P.fdir[c] + cs * P.sdir[c] +
                   cn * P.ndir[c];
        double R = sqrt(bg_dot3(pos, pos));
#pragma unroll
        for (int c = 0; c < 3; ++c) d[c] = pos[c] / R;
        double omega = px * px * bg_dot3(P.ndir, pos) / (R * R * R);
        double cap = 1.0;
        if (a.thickness > 0.0) {
          double L = a.atten * bg_dot3(d, P.ndir);
          cap = exp(-t * a.dt / L) - exp(-(t + 1) * a.dt / L);
        }
        for (int g = 0; g < b.n_groups; ++g) {
          const double *dir = s_grp + 9 * g;
          double v[3] = {d[0] - dir[0], d[1] - dir[1], d[2] - dir[2]};
          double half = 0.5 * sqrt(bg_dot3(v, v));  // sin(theta)
          // Kahn: cos 2psi sin^2 2theta = (d.E')^2 - (d.B')^2 for unit d
          double c2 = bg_dot3(d, dir), x = bg_dot3(d, dir + 3),
                 y = bg_dot3(d, dir + 6);
          double pol = 0.5 * (1.0 + c2 * c2 - a.kahn64 * (x * x - y * y));
          const int k0 = s_rng[2 * g], k1 = k0 + s_rng[2 * g + 1];
          double gsum;
          if (F64) {
            const double s0 = s_k64[0], sn = s_k64[2 * (n - 1)];
            int jk = -1;
            gsum = 0.0;
            for (int k = k0; k < k1; ++k) {
              double st = half * s_src64[2 * k];
              double Fb;
              if (st <= s0) {
                Fb = s_k64[1];
              } else if (st >= sn) {
                Fb = s_k64[2 * (n - 1) + 1];
              } else {
                if (jk < 0)
                  jk = bg_search(s_k64, 2, n, st);
                else
                  while (s_k64[2 * (jk + 1)] <= st) ++jk;
                const double *kn = s_k64 + 2 * jk;
                double tt = (st - kn[0]) / (kn[2] - kn[0]);
                Fb = kn[1] + tt * (kn[3] - kn[1]);
              }
              gsum += Fb * Fb * s_src64[2 * k + 1];
            }
          } else {
            const float halff = (float)half;
            const float s0 = s_k32[0], sn = s_k32[3 * (n - 1)];
            int jk = -1;
            Kahan ks;
            for (int k = k0; k < k1; ++k) {
              float st = halff * s_src32[2 * k];
              float Fb;
              if (st <= s0) {
                Fb = s_k32[1];
              } else if (st >= sn) {
                Fb = s_k32[3 * (n - 1) + 1];
              } else {
                if (jk < 0)
                  jk = bg_search(s_k32, 3, n, st);
                else
                  while (s_k32[3 * (jk + 1)] <= st) ++jk;
                const float *kn = s_k32 + 3 * jk;
                Fb = fmaf(st - kn[0], kn[2], kn[1]);
              }
              ks.add(Fb * Fb * s_src32[2 * k + 1]);
            }
            gsum = (double)ks.value();
          }
          acc += gsum * (cap * pol * omega);
        }
      }
  // addArray: the pixel's value is rounded first, then added (no FMA)
  a.image[gp] = __dadd_rn(a.image[gp], __dmul_rn(b.prefactor, acc));
}

size_t background_smem_bytes(const BgArgs &b, bool f64) {
  size_t bytes = (size_t)b.n_groups * 9 * sizeof(double) +
                 (size_t)b.n_groups * 2 * sizeof(int);
  if (f64)
    bytes += ((size_t)b.n_knots * 2 + (size_t)b.geo.S * 2) * sizeof(double);
  else
    bytes += ((size_t)b.n_knots * 3 + (size_t)b.geo.S * 2) * sizeof(float);
  return bytes;
}

cudaError_t launch_background(const BgArgs &b, bool f64, cudaStream_t st) {
  if (b.geo.n_tiles <= 0) return cudaSuccess;
  size_t smem = background_smem_bytes(b, f64);
  void (*kern)(BgArgs) = f64 ? background_kernel<1> : background_kernel<0>;
  cudaError_t e = cudaFuncSetAttribute(
      kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)b.geo.n_tiles, kTileThreads, smem, st>>>(b);
  return cudaGetLastError();
}

}  // namespace nbgb
