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
#include "nbgb_internal.cuh"

namespace nbgb {

__device__ __forceinline__ double dot3d_m(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// double-float dot product of A (hi, lo) with v (hi, lo)
__device__ __forceinline__ void ff_dot3(const float *Ah, const float *Al,
                                        const float *vh, const float *vl,
                                        float &gh, float &gl) {
  float p0, e0, p1, e1, p2, e2;
  two_prod(Ah[0], vh[0], p0, e0);
  two_prod(Ah[1], vh[1], p1, e1);
  two_prod(Ah[2], vh[2], p2, e2);
  float s, t, s2, t2;
  two_sum(p0, p1, s, t);
  two_sum(s, p2, s2, t2);
  float lo = e0 + e1 + e2 + t + t2;
  lo = fmaf(Ah[0], vl[0], lo);
  lo = fmaf(Ah[1], vl[1], lo);
  lo = fmaf(Ah[2], vl[2], lo);
  lo = fmaf(Al[0], vh[0], lo);
  lo = fmaf(Al[1], vh[1], lo);
  lo = fmaf(Al[2], vh[2], lo);
  fast_two_sum(s2, lo, gh, gl);
}

// fractional offset of h = G (u0 + delta) - E relative to its nearest
// integer, given r = G u0 - n0 (double-float).  Returns f = fh + fl and the
// integer shift nf (h = n0 + nf + f).
template <int HASDIV>
__device__ __forceinline__ void frac_ff(float Gh, float Gl, float rh, float rl,
                                        float dh, float dl, float Eh, float El,
                                        float &fh, float &fl, float &nf) {
  float p, pe, t, te;
  two_prod(Gh, dh, p, pe);
  two_sum(p, rh, t, te);
  float lo = pe + te + rl;
  if (HASDIV) {
    float t3, te3;
    two_sum(t, -Eh, t3, te3);
    t = t3;
    lo = lo + te3 - El;
  }
  lo = fmaf(Gh, dl, lo);
  lo = fmaf(Gl, dh, lo);
  nf = rintf(t);
  float t2 = __fsub_rn(t, nf);  // exact
  fh = __fadd_rn(t2, lo);
  fl = __fsub_rn(lo, __fsub_rn(fh, t2));
}

template <int INTERP>
__device__ __forceinline__ float fcell_f32(const SpotArgs &a, const int n[3],
                                           const float fr[3]) {
  if (INTERP == 1) {
    int fl[3];
    float x[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      int neg = fr[c] < 0.f;
      fl[c] = n[c] - neg;
      x[c] = neg ? 1.f + fr[c] : fr[c];
    }
    // the 4x4x4 stencil fl-1 .. fl+2 must lie inside the table
    if (fl[0] >= 1 && fl[0] + 2 < a.hn[0] && fl[1] >= 1 &&
        fl[1] + 2 < a.hn[1] && fl[2] >= 1 && fl[2] + 2 < a.hn[2]) {
      float wh[4], wk[4], wl[4];
      lagrange4(x[0], wh);
      lagrange4(x[1], wk);
      lagrange4(x[2], wl);
      const float *base =
          a.F + ((long long)(fl[0] - 1) * a.hn[1] + (fl[1] - 1)) * a.hn[2] +
          (fl[2] - 1);
      float sum = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float si = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float *row = base + ((long long)i * a.hn[1] + j) * a.hn[2];
          float sj = wl[0] * __ldg(row);
          sj = fmaf(wl[1], __ldg(row + 1), sj);
          sj = fmaf(wl[2], __ldg(row + 2), sj);
          sj = fmaf(wl[3], __ldg(row + 3), sj);
          si = fmaf(wk[j], sj, si);
        }
        sum = fmaf(wh[i], si, sum);
      }
      return sum;
    }
  }
  if ((unsigned)n[0] < (unsigned)a.hn[0] && (unsigned)n[1] < (unsigned)a.hn[1] &&
      (unsigned)n[2] < (unsigned)a.hn[2])
    return __ldg(a.F + ((long long)n[0] * a.hn[1] + n[1]) * a.hn[2] + n[2]);
  return a.defF;
}

// MODE 0: NB_MIXED, MODE 1: NB_F32
template <int SHAPE, int INTERP, int MODE, int HASDIV>
__global__ void __launch_bounds__(kTileThreads, 4)
    spots_mixed_kernel(SpotArgs a) {
  extern __shared__ float smf[];
  float *s_axh = smf;
  float *s_axl = smf + a.PM * 9;
  float *s_src = smf + 2 * a.PM * 9;
  for (int i = threadIdx.x; i < a.PM * 9; i += blockDim.x) {
    s_axh[i] = a.axh[i];
    s_axl[i] = a.axl[i];
  }
  for (int i = threadIdx.x; i < a.S * SRC32_STRIDE; i += blockDim.x)
    s_src[i] = a.src32[i];
  __syncthreads();

  long long item = a.pixlist ? (long long)blockIdx.x * blockDim.x + threadIdx.x
                             : (long long)blockIdx.x;
  long long gp;
  int q, s, f;
  if (!map_pixel(a, item, threadIdx.x, gp, q, s, f)) return;
  const DevPanel &P = a.panels[q];
  const double px = P.px;
  const int os = a.os;
  const float kahn = a.kahn;
  const float cutg = kGaussCut * 0.63f;
  double total = 0.0;
  unsigned evals = 0;  // terms evaluated (not skipped by the underflow cut)

  for (int i = 0; i < os; ++i) {
    for (int j = 0; j < os; ++j) {
      for (int t = 0; t < a.T; ++t) {
        // ---- per subpixel / layer: geometry
        float df[3], vh[3], vl[3], omega, cap = 1.f;
        if (MODE == 0) {
          double cf = (f + (i + 0.5) / os) * px, cs = (s + (j + 0.5) / os) * px,
                 cn = t * a.dt;
          double pos[3], d[3];
#pragma unroll
          for (int c = 0; c < 3; ++c)
            pos[c] = P.origin[c] + cf * P.fdir[c] + cs * P.sdir[c] +
                     cn * P.ndir[c];
          double R = sqrt(dot3d_m(pos, pos));
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            d[c] = pos[c] / R;
            df[c] = (float)d[c];
            double v = d[c] - a.i0[c];
            vh[c] = (float)v;
            vl[c] = (float)(v - (double)vh[c]);
          }
          omega = (float)(px * px * dot3d_m(P.ndir, pos) / (R * R * R));
        } else {
          float cf = (f + (i + 0.5f) / os) * (float)px,
                cs = (s + (j + 0.5f) / os) * (float)px, cn = t * (float)a.dt;
          float pos[3];
#pragma unroll
          for (int c = 0; c < 3; ++c)
            pos[c] = (float)P.origin[c] + cf * (float)P.fdir[c] +
                     cs * (float)P.sdir[c] + cn * (float)P.ndir[c];
          float R = sqrtf(pos[0] * pos[0] + pos[1] * pos[1] + pos[2] * pos[2]);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            df[c] = pos[c] / R;
            vh[c] = df[c] - (float)a.i0[c];
            vl[c] = 0.f;
          }
          float nd = pos[0] * (float)P.ndir[0] + pos[1] * (float)P.ndir[1] +
                     pos[2] * (float)P.ndir[2];
          omega = (float)px * (float)px * nd / (R * R * R);
        }
        if (a.thickness > 0.0) {
          float rho = df[0] * (float)P.ndir[0] + df[1] * (float)P.ndir[1] +
                      df[2] * (float)P.ndir[2];
          float L = (float)a.atten * rho, dtf = (float)a.dt;
          cap = expf(-t * dtf / L) - expf(-(t + 1) * dtf / L);
        }
        float scal = omega * cap;
        if (!HASDIV) {
          float c2 = df[0] * (float)a.i0[0] + df[1] * (float)a.i0[1] +
                     df[2] * (float)a.i0[2];
          float x = df[0] * (float)a.e0[0] + df[1] * (float)a.e0[1] +
                    df[2] * (float)a.e0[2];
          float y = df[0] * (float)a.b0[0] + df[1] * (float)a.b0[1] +
                    df[2] * (float)a.b0[2];
          scal *= 0.5f * (1.f + c2 * c2 - kahn * (x * x - y * y));
        }
        Kahan acc;
        for (int pm = 0; pm < a.PM; ++pm) {
          // ---- per (subpixel, phi x mosaic): G = A.(d - i0), r = u0 G - n0
          const float *Ah = s_axh + pm * 9, *Al = s_axl + pm * 9;
          float Gh[3], Gl[3], rh[3], rl[3], n0[3];
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            if (MODE == 0) {
              ff_dot3(Ah + 3 * x, Al + 3 * x, vh, vl, Gh[x], Gl[x]);
              float qh, qe;
              two_prod(Gh[x], a.u0h, qh, qe);
              float ql = fmaf(Gh[x], a.u0l, fmaf(Gl[x], a.u0h, qe));
              n0[x] = rintf(qh);
              two_sum(__fsub_rn(qh, n0[x]), ql, rh[x], rl[x]);
            } else {
              Gh[x] = Ah[3 * x] * vh[0] + Ah[3 * x + 1] * vh[1] +
                      Ah[3 * x + 2] * vh[2];
              Gl[x] = 0.f;
              rh[x] = rl[x] = n0[x] = 0.f;
            }
          }
          for (int k = 0; k < a.S; ++k) {
            const float *src = s_src + k * SRC32_STRIDE;
            float fr[3], frl[3];
            int n[3];
#pragma unroll
            for (int x = 0; x < 3; ++x) {
              float Eh = 0.f, El = 0.f;
              if (HASDIV) {
                size_t e = ((size_t)pm * a.S + k) * 3 + x;
                Eh = __ldg(a.divh + e);
                El = __ldg(a.divl + e);
              }
              float nf;
              if (MODE == 0) {
                frac_ff<HASDIV>(Gh[x], Gl[x], rh[x], rl[x], src[SRC32_DH],
                                src[SRC32_DL], Eh, El, fr[x], frl[x], nf);
              } else {
                // NB_F32: h = G u_k - E in plain FP32 (src[DL] holds u_k)
                float h = Gh[x] * src[SRC32_DL] - Eh;
                nf = rintf(h);
                fr[x] = h - nf;
                frl[x] = 0.f;
              }
              n[x] = __float2int_rn(n0[x] + nf) - a.hmin[x];
            }
            float fl2;
            if (SHAPE == 1) {
              float rad2 = a.N[0] * a.N[0] * fr[0] * fr[0];
              rad2 = fmaf(a.N[1] * a.N[1], fr[1] * fr[1], rad2);
              rad2 = fmaf(a.N[2] * a.N[2], fr[2] * fr[2], rad2);
              if (rad2 > cutg) continue;
              fl2 = a.N6 * expf(-2.f * rad2 * (1.f / 0.63f));
              ++evals;
            } else {
              float nump = 1.f, denp = 1.f;
#pragma unroll
              for (int x = 0; x < 3; ++x) {
                float yh, yr;
                if (MODE == 0) {
                  float ye;
                  two_prod(a.N[x], fr[x], yh, ye);
                  float yl = fmaf(a.N[x], frl[x], ye);
                  yr = __fsub_rn(yh, rintf(yh)) + yl;
                } else {
                  yh = a.N[x] * fr[x];
                  yr = yh - rintf(yh);
                }
                float num, den;
                if (fabsf(fr[x]) < 1e-9f) {
                  num = a.N[x];
                  den = 1.f;
                } else {
                  num = sinpi_reduced(yr);
                  den = sinpi_reduced(fr[x]);
                }
                nump *= num;
                denp *= den;
              }
              float ratio = nump / denp;
              fl2 = ratio * ratio;
              ++evals;
            }
            float fc = fcell_f32<INTERP>(a, n, fr);
            float w = src[SRC32_W];
            if (HASDIV) {
              const float *dir = src + SRC32_DIR, *ev = src + SRC32_E,
                          *bv = src + SRC32_B;
              float c2 = df[0] * dir[0] + df[1] * dir[1] + df[2] * dir[2];
              float x = df[0] * ev[0] + df[1] * ev[1] + df[2] * ev[2];
              float y = df[0] * bv[0] + df[1] * bv[1] + df[2] * bv[2];
              w *= 0.5f * (1.f + c2 * c2 - kahn * (x * x - y * y));
            }
            acc.add(fc * fc * fl2 * w);
          }
        }
        total += (double)scal * acc.value();
      }
    }
  }
  a.image[gp] += a.prefactor * total;
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

cudaError_t launch_spots_mixed(const SpotArgs &a, int precision,
                               cudaStream_t st) {
  size_t smem = (size_t)(2 * a.PM * 9 + a.S * SRC32_STRIDE) * sizeof(float);
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
