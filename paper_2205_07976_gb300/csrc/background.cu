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
// from the previous one.  The F64 form is FP64 throughout; the mixed form
// is FP32 after the pixel's corner, with compensated sums per group and
// per pixel.
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

// ------------------------------------------------------------ FP64 form

__global__ void __launch_bounds__(kTileThreads)
    background_f64_kernel(BgArgs b) {
  const SpotArgs &a = b.geo;
  extern __shared__ double smd[];
  double *s_grp = smd;                     // [G][9] dir, E', B'
  double *s_k64 = s_grp + b.n_groups * 9;  // [n][2] stol, F
  double *s_src = s_k64 + 2 * b.n_knots;   // [S][2] 1/lambda, w
  int *s_rng = (int *)(s_src + 2 * a.S);   // [G][2]
  for (int i = threadIdx.x; i < b.n_groups * 9; i += blockDim.x)
    s_grp[i] = b.grp64[i];
  for (int i = threadIdx.x; i < 2 * b.n_groups; i += blockDim.x)
    s_rng[i] = b.grp_range[i];
  for (int i = threadIdx.x; i < 2 * b.n_knots; i += blockDim.x)
    s_k64[i] = b.knots64[i];
  for (int i = threadIdx.x; i < 2 * a.S; i += blockDim.x)
    s_src[i] = b.src64[i];
  __syncthreads();

  long long gp;
  int q, s, f;
  if (!map_pixel(a, (long long)blockIdx.x, threadIdx.x, gp, q, s, f)) return;
  const DevPanel &P = a.panels[q];
  const double px = P.px;
  const int os = a.os, n = b.n_knots;
  const double s0 = s_k64[0], sn = s_k64[2 * (n - 1)];
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
          int jk = -1;
          double gsum = 0.0;
          for (int k = k0; k < k1; ++k) {
            double st = half * s_src[2 * k];
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
            gsum += Fb * Fb * s_src[2 * k + 1];
          }
          acc += gsum * (cap * pol * omega);
        }
      }
  // addArray: the pixel's value is rounded first, then added (no FMA)
  gp = nb_idx(a.check, NB_SITE_IMAGE, gp, a.npix);
  a.image[gp] = __dadd_rn(a.image[gp], __dmul_rn(b.prefactor, acc));
}

// ----------------------------------------------------------- mixed form
//
// Everything after the pixel's corner is FP32.  |d - i| is formed without
// cancellation near the direct beam: with p = pos . i and p_perp =
// |pos x i|, d - i has the components (p - R)/R = -p_perp^2 / (R (R + p))
// along i and p_perp / R across it.  The current interval (start, F,
// slope, end) is one float4 in registers; the held ends are intervals of
// slope 0, so each source costs one compare to stay or walk on.

__device__ __forceinline__ float bg_dot3f(const float *a, const float *b) {
  return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}

__global__ void __launch_bounds__(kTileThreads)
    background_mixed_kernel(BgArgs b) {
  const SpotArgs &a = b.geo;
  extern __shared__ float4 smq[];
  // intervals e = 0..n: e = 0 holds F_0 below stol_0, e = j + 1 is the
  // knot interval [stol_j, stol_j+1), e = n holds F_n-1 from stol_n-1 on;
  // each is (start, F at start, slope, end)
  float4 *s_k4 = smq;                                 // [n + 1]
  float2 *s_src = (float2 *)(s_k4 + b.n_knots + 1);   // [S] 1/lambda, w
  float *s_grp = (float *)(s_src + a.S);              // [G][9]
  int *s_rng = (int *)(s_grp + 9 * b.n_groups);       // [G][2]
  const int n = b.n_knots;
  const float inf = __int_as_float(0x7f800000);
  for (int e = threadIdx.x; e <= n; e += blockDim.x) {
    float4 v;
    if (e == 0) {
      v = make_float4(b.knots32[0], b.knots32[1], 0.f, b.knots32[0]);
    } else if (e == n) {
      const float *kn = b.knots32 + 3 * (n - 1);
      v = make_float4(kn[0], kn[1], 0.f, inf);
    } else {
      const float *kn = b.knots32 + 3 * (e - 1);
      v = make_float4(kn[0], kn[1], kn[2], kn[3]);
    }
    s_k4[e] = v;
  }
  for (int i = threadIdx.x; i < a.S; i += blockDim.x)
    s_src[i] = make_float2(b.src32[2 * i], b.src32[2 * i + 1]);
  for (int i = threadIdx.x; i < b.n_groups * 9; i += blockDim.x)
    s_grp[i] = (float)b.grp64[i];
  for (int i = threadIdx.x; i < 2 * b.n_groups; i += blockDim.x)
    s_rng[i] = b.grp_range[i];
  __syncthreads();

  long long gp;
  int q, s, f;
  if (!map_pixel(a, (long long)blockIdx.x, threadIdx.x, gp, q, s, f)) return;
  const DevPanel &P = a.panels[q];
  const double px = P.px;
  const int os = a.os;
  const float s_first = s_k4[0].x, s_last = s_k4[n].x;
  const float kahn = (float)a.kahn64;
  const float nd[3] = {(float)P.ndir[0], (float)P.ndir[1], (float)P.ndir[2]};
  const float px2 = (float)(px * px);
  const float dtf = (float)a.dt, attf = (float)a.atten;
  // the pixel's corner in FP64, the subpixel offsets from it in FP32
  float base[3], fd[3], sd[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    base[c] = (float)(P.origin[c] + f * px * P.fdir[c] + s * px * P.sdir[c]);
    fd[c] = (float)P.fdir[c];
    sd[c] = (float)P.sdir[c];
  }
  const float sub = (float)(px / os);
  Kahan acc;  // over (subpixel, layer, group) of the group sums
  for (int i = 0; i < os; ++i)
    for (int j = 0; j < os; ++j)
      for (int t = 0; t < a.T; ++t) {
        const float cf = (i + 0.5f) * sub, cs = (j + 0.5f) * sub,
                    cn = t * dtf;
        float pos[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          pos[c] = fmaf(cf, fd[c], fmaf(cs, sd[c], fmaf(cn, nd[c], base[c])));
        float R2 = bg_dot3f(pos, pos);
        float rinv = rsqrtf(R2), R = R2 * rinv;
        float pn = bg_dot3f(nd, pos);
        float omega = px2 * pn * (rinv * rinv * rinv);
        float cap = 1.f;
        if (a.thickness > 0.0) {
          float L = attf * pn * rinv;
          cap = __expf(-t * dtf / L) - __expf(-(t + 1) * dtf / L);
        }
        float fac = omega * cap;
        for (int g = 0; g < b.n_groups; ++g) {
          const float *dir = s_grp + 9 * g;
          float p = bg_dot3f(pos, dir);
          float cx = pos[1] * dir[2] - pos[2] * dir[1],
                cy = pos[2] * dir[0] - pos[0] * dir[2],
                cz = pos[0] * dir[1] - pos[1] * dir[0];
          float pp2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
          float dd2;  // |d - i|^2
          if (p > 0.f) {
            float along = pp2 / (R * (R + p));
            dd2 = fmaf(along, along, pp2 * (rinv * rinv));
          } else {
            float vx = pos[0] * rinv - dir[0], vy = pos[1] * rinv - dir[1],
                  vz = pos[2] * rinv - dir[2];
            dd2 = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
          }
          const float half = 0.5f * sqrtf(dd2);  // sin(theta)
          float c2 = p * rinv, x = bg_dot3f(pos, dir + 3) * rinv,
                y = bg_dot3f(pos, dir + 6) * rinv;
          float pol = 0.5f * (1.f + c2 * c2 - kahn * (x * x - y * y));
          const int k0 = s_rng[2 * g], k1 = k0 + s_rng[2 * g + 1];
          if (k0 >= k1) continue;
          // interval of the group's first (smallest) stol, then walk
          int e;
          {
            const float st = half * s_src[k0].x;
            e = st < s_first ? 0
                : st >= s_last ? n
                               : 1 + bg_search(&s_k4[1].x, 4, n, st);
          }
          float4 kb = s_k4[e];
          // the source terms of one block of up to 32 sources go into four
          // plain FP32 chains (at most 8 positive terms each, so the block
          // sum is within 10 ulp); the blocks are added compensated, which
          // keeps the bound independent of the number of sources
          auto term = [&](int k) {
            const float2 uw = s_src[k];
            const float st = half * uw.x;
            while (st >= kb.w) kb = s_k4[++e];
            const float Fb = fmaf(st - kb.x, kb.z, kb.y);
            return make_float2(Fb * uw.y, Fb);
          };
          Kahan ks;
          for (int k = k0; k < k1;) {
            const int kend = min(k + 32, k1);
            float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
            for (; k + 4 <= kend; k += 4) {
              float2 t0 = term(k);
              c0 = fmaf(t0.x, t0.y, c0);
              float2 t1 = term(k + 1);
              c1 = fmaf(t1.x, t1.y, c1);
              float2 t2 = term(k + 2);
              c2 = fmaf(t2.x, t2.y, c2);
              float2 t3 = term(k + 3);
              c3 = fmaf(t3.x, t3.y, c3);
            }
            for (; k < kend; ++k) {
              float2 t0 = term(k);
              c0 = fmaf(t0.x, t0.y, c0);
            }
            ks.add((c0 + c1) + (c2 + c3));
          }
          acc.add(__fsub_rn(ks.s, ks.c) * (fac * pol));
        }
      }
  // addArray: the pixel's value is rounded first, then added (no FMA)
  gp = nb_idx(a.check, NB_SITE_IMAGE, gp, a.npix);
  a.image[gp] = __dadd_rn(a.image[gp], __dmul_rn(b.prefactor, acc.value()));
}

size_t background_smem_bytes(const BgArgs &b, bool f64) {
  if (f64)
    return ((size_t)b.n_groups * 9 + (size_t)b.n_knots * 2 +
            (size_t)b.geo.S * 2) * sizeof(double) +
           (size_t)b.n_groups * 2 * sizeof(int);
  return (size_t)(b.n_knots + 1) * sizeof(float4) + (size_t)b.geo.S * 8 +
         (size_t)b.n_groups * 9 * sizeof(float) +
         (size_t)b.n_groups * 2 * sizeof(int);
}

cudaError_t launch_background(const BgArgs &b, bool f64, cudaStream_t st) {
  if (b.geo.n_tiles <= 0) return cudaSuccess;
  size_t smem = background_smem_bytes(b, f64);
  void (*kern)(BgArgs) = f64 ? background_f64_kernel : background_mixed_kernel;
  cudaError_t e = cudaFuncSetAttribute(
      kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)b.geo.n_tiles, kTileThreads, smem, st>>>(b);
  return cudaGetLastError();
}

}  // namespace nbgb
