// adjoint.cu -- gradients of a scalar image loss through the Bragg-spot sum
// (the refinement loop of x-ray tracing, Sec. II: crystal parameters are
// refined until the simulated image matches the measured one), and the
// Poisson image loss itself.
//
// The crystal is parametrised as lab axes = rows of Rx(tx) Ry(ty) Rz(tz) U
// diag(a, b, c) (orthorhombic cell, fixed orientation U, three small
// rotations), Gaussian F_latt with Na, Nb, Nc, an overall scale and the
// structure-factor table (nearest or tricubic lookup).  Given w_p = dL/dI_p for every
// pixel, the kernel recomputes every step of the forward sum (nothing is
// stored between passes) and accumulates
//   dL/dθ_r  = Σ_p w_p K scale Σ_steps term · Σ_x dlog(F_latt^2)/df_x · dh_x/dθ_r
//   dL/dN_x  = Σ_p w_p K scale Σ_steps term · (2/N_x − 4 N_x f_x^2/0.63)
//   dL/dscale = Σ_p w_p I_p / scale
//   dL/dF[h0] += w_p K scale · 2 F_cell F_latt^2 w_k cap pol ω    (scatter-add)
// with dh_x/dθ_r = (∂A_x/∂θ_r) · (d − i)/λ and dlog(F_latt^2)/df_x =
// −4 N_x^2 f_x / 0.63; with tricubic lookup F_cell also depends on h (the
// derivative of the Lagrange weights) and dL/dF is spread over the 64
// stencil entries with the interpolation weights.  The per-step arithmetic
// is the FP32-mixed form of the forward kernel (double-float fractional
// offsets); the ten scalar sums
// go per thread into FP64, per block into a partial row, and a second
// kernel adds the rows in a fixed order.
#include "mixed_common.cuh"

namespace nbgb {

struct AdjointArgs {
  SpotArgs a;
  const float *dax;      // [PM][6][9] d(rotated axes)/d(tx,ty,tz,a,b,c)
  const double *dLdI;    // [npix]
  double *gradF;         // [nh*nk*nl], accumulated into
  double *partials;      // [blocks][kGradN]
  double kc;             // r_e^2 fluence / (os^2 M Phi)
  double scale;
};

constexpr int kGradN = 10;

// derivatives of the 4-point Lagrange weights (nodes -1, 0, 1, 2) at x
__device__ __forceinline__ void lagrange4_deriv(float x, float w[4]) {
  float x2 = x * x;
  w[0] = -(3.f * x2 - 6.f * x + 2.f) * (1.f / 6.f);
  w[1] = (3.f * x2 - 4.f * x - 1.f) * 0.5f;
  w[2] = -(3.f * x2 - 2.f * x - 2.f) * 0.5f;
  w[3] = (3.f * x2 - 1.f) * (1.f / 6.f);
}

template <int HASF, int INTERP>
__global__ void __launch_bounds__(kTileThreads, INTERP ? 3 : 4)
    spots_adjoint_kernel(AdjointArgs g) {
  const SpotArgs &a = g.a;
  extern __shared__ float smf[];
  float *s_axh = smf;
  float *s_axl = smf + a.PM * 9;
  float *s_src = smf + 2 * a.PM * 9;
  float *s_dax = s_src + a.S * SRC32_STRIDE;
  for (int i = threadIdx.x; i < a.PM * 9; i += blockDim.x) {
    s_axh[i] = a.axh[i];
    s_axl[i] = a.axl[i];
  }
  for (int i = threadIdx.x; i < a.S * SRC32_STRIDE; i += blockDim.x)
    s_src[i] = a.src32[i];
  for (int i = threadIdx.x; i < a.PM * 54; i += blockDim.x)
    s_dax[i] = g.dax[i];
  __syncthreads();
  // tricubic dL/dF: the terms of a thread near one lattice point n use
  // stencils starting at n-2 or n-1 along each axis, all inside the 5x5x5
  // nodes n-2 .. n+2.  The thread sums their weighted contributions there,
  // in its own column of shared memory (FP32), and adds the touched nodes
  // to the FP64 gradient when n changes and at the end: far fewer global
  // atomics than 64 per term.
  // [125][kTileThreads] after the tables (dynamic shared memory)
  float (*s_facc)[kTileThreads] =
      reinterpret_cast<float (*)[kTileThreads]>(s_dax + a.PM * 54);
  long long near_idx = -1;  // nearest lookup: the entry being summed
  double near_sum = 0.0;
  int held[3] = {0, 0, 0};  // the lattice point held (table-relative)
  bool holding = false;
  auto flush_node = [&]() {
    if (!holding) return;
    for (int e = 0; e < 125; ++e) {
      const float v = s_facc[e][threadIdx.x];
      if (v == 0.f) continue;  // untouched (may lie outside the table)
      s_facc[e][threadIdx.x] = 0.f;
      const int i = e / 25, j = (e / 5) % 5, k = e % 5;
      atomicAdd(g.gradF + ((long long)(held[0] - 2 + i) * a.hn[1] +
                           (held[1] - 2 + j)) * a.hn[2] + (held[2] - 2 + k),
                (double)v);
    }
    holding = false;
  };
  if (INTERP && HASF)
    for (int e = 0; e < 125; ++e) s_facc[e][threadIdx.x] = 0.f;

  double gsum[kGradN];
#pragma unroll
  for (int r = 0; r < kGradN; ++r) gsum[r] = 0.0;

  long long item = a.pixlist ? (long long)blockIdx.x * blockDim.x + threadIdx.x
                             : (long long)blockIdx.x;
  long long gp;
  int q, s, f;
  if (map_pixel(a, item, threadIdx.x, gp, q, s, f)) {
    const DevPanel &P = a.panels[q];
    const int os = a.os;
    const float kahn = a.kahn;
    const float cutg = kGaussCut * 0.63f;
    const double wp = g.dLdI[gp];
    const double wks = wp * g.kc * g.scale;
    const float N2[3] = {a.N[0] * a.N[0], a.N[1] * a.N[1], a.N[2] * a.N[2]};
    double tot[kGradN];
#pragma unroll
    for (int r = 0; r < kGradN; ++r) tot[r] = 0.0;
    for (int i = 0; i < os; ++i)
      for (int j = 0; j < os; ++j)
        for (int t = 0; t < a.T; ++t) {
          float vh[3], vl[3], v32[3], df[3], omega;
          unit_geometry_ff(a, P, s, f, i, j, t, vh, vl, df, omega);
#pragma unroll
          for (int c = 0; c < 3; ++c) v32[c] = vh[c];
          float cap = 1.f;
          if (a.dtff[0] > 0.f) {
            float rho = df[0] * P.ffn[0][0] + df[1] * P.ffn[1][0] +
                        df[2] * P.ffn[2][0];
            float L = a.attenf * rho, dtf = a.dtff[0];
            cap = expf(-t * dtf / L) - expf(-(t + 1) * dtf / L);
          }
          float c2 = df[0] * a.i0ff[0][0] + df[1] * a.i0ff[1][0] +
                     df[2] * a.i0ff[2][0],
                xe = df[0] * a.e0f[0] + df[1] * a.e0f[1] + df[2] * a.e0f[2],
                ye = df[0] * a.b0f[0] + df[1] * a.b0f[1] + df[2] * a.b0f[2];
          float scal = omega * cap * 0.5f *
                       (1.f + c2 * c2 - kahn * (xe * xe - ye * ye));
          const double fscal = wks * (double)scal;  // for the F scatter
          Kahan acc0;
          float acc[9];
#pragma unroll
          for (int r = 0; r < 9; ++r) acc[r] = 0.f;
          for (int pm = 0; pm < a.PM; ++pm) {
            const float *Ah = s_axh + pm * 9, *Al = s_axl + pm * 9;
            float Gh[3], Gl[3], rq[3], rl[3], n0[3];
#pragma unroll
            for (int x = 0; x < 3; ++x) {
              ff_dot3(Ah + 3 * x, Al + 3 * x, vh, vl, Gh[x], Gl[x]);
              float qh, qe;
              two_prod(Gh[x], a.u0h, qh, qe);
              float ql = fmaf(Gh[x], a.u0l, fmaf(Gl[x], a.u0h, qe));
              n0[x] = rintf(qh);
              float rh, rl0;
              two_sum(__fsub_rn(qh, n0[x]), ql, rh, rl0);
              rq[x] = __fmul_rn(rintf(__fmul_rn(rh, 2097152.f)),
                                1.f / 2097152.f);
              rl[x] = rl0 + __fsub_rn(rh, rq[x]);
            }
            // dG[r][x] = dA_pm[r][x] . (d - i0)
            float dG[6][3];
            const float *dA = s_dax + pm * 54;
#pragma unroll
            for (int r = 0; r < 6; ++r)
#pragma unroll
              for (int x = 0; x < 3; ++x)
                dG[r][x] = dA[r * 9 + 3 * x] * v32[0] +
                           dA[r * 9 + 3 * x + 1] * v32[1] +
                           dA[r * 9 + 3 * x + 2] * v32[2];
            for (int k = 0; k < a.S; ++k) {
              const float *src = s_src + k * SRC32_STRIDE;
              const float dh = src[SRC32_DH], dl = src[SRC32_DL];
              float fr[3], nf[3];
#pragma unroll
              for (int x = 0; x < 3; ++x) {
                float tq = fmaf(Gh[x], dh, rq[x]);
                nf[x] = rintf(tq);
                fr[x] = tq - nf[x];
              }
              float rad2 = N2[0] * fr[0] * fr[0];
              rad2 = fmaf(N2[1] * fr[1], fr[1], rad2);
              rad2 = fmaf(N2[2] * fr[2], fr[2], rad2);
              if (rad2 > cutg) continue;
#pragma unroll
              for (int x = 0; x < 3; ++x) {
                float sx = fmaf(Gh[x], dh, __fsub_rn(rq[x], nf[x]));
                fr[x] = sx + fmaf(Gh[x], dl, fmaf(Gl[x], dh, rl[x]));
              }
              rad2 = N2[0] * fr[0] * fr[0];
              rad2 = fmaf(N2[1] * fr[1], fr[1], rad2);
              rad2 = fmaf(N2[2] * fr[2], fr[2], rad2);
              float fl2 = a.N6 * expf(-2.f * rad2 * (1.f / 0.63f));
              int n[3];
#pragma unroll
              for (int x = 0; x < 3; ++x)
                n[x] = __float2int_rn(n0[x] + nf[x]) - a.hmin[x];
              bool inside = (unsigned)n[0] < (unsigned)a.hn[0] &&
                            (unsigned)n[1] < (unsigned)a.hn[1] &&
                            (unsigned)n[2] < (unsigned)a.hn[2];
              long long fidx =
                  inside ? ((long long)n[0] * a.hn[1] + n[1]) * a.hn[2] + n[2]
                         : -1;
              float fc, dfc[3] = {0.f, 0.f, 0.f};
              // tricubic: value and gradient of the interpolant, and the
              // stencil (its weights feed the structure-factor gradient)
              bool tri = false;
              int fl[3];
              float wv[3][4];
              if (INTERP == 1) {
                float xs[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  int neg = fr[c] < 0.f;
                  fl[c] = n[c] - neg;
                  xs[c] = neg ? 1.f + fr[c] : fr[c];
                }
                tri = fl[0] >= 1 && fl[0] + 2 < a.hn[0] && fl[1] >= 1 &&
                      fl[1] + 2 < a.hn[1] && fl[2] >= 1 && fl[2] + 2 < a.hn[2];
                if (tri) {
                  float wd[3][4];
#pragma unroll
                  for (int c = 0; c < 3; ++c) {
                    lagrange4(xs[c], wv[c]);
                    lagrange4_deriv(xs[c], wd[c]);
                  }
                  fc = 0.f;
                  for (int i = 0; i < 4; ++i)
                    for (int j = 0; j < 4; ++j) {
                      const float *row =
                          a.F + ((long long)(fl[0] - 1 + i) * a.hn[1] +
                                 (fl[1] - 1 + j)) * a.hn[2] + (fl[2] - 1);
#pragma unroll
                      for (int k = 0; k < 4; ++k) {
                        float Fv = __ldg(row + k);
                        float wij = wv[0][i] * wv[1][j];
                        fc = fmaf(wij * wv[2][k], Fv, fc);
                        dfc[0] = fmaf(wd[0][i] * wv[1][j] * wv[2][k], Fv, dfc[0]);
                        dfc[1] = fmaf(wv[0][i] * wd[1][j] * wv[2][k], Fv, dfc[1]);
                        dfc[2] = fmaf(wij * wd[2][k], Fv, dfc[2]);
                      }
                    }
                }
              }
              if (!tri) fc = inside ? __ldg(a.F + fidx) : a.defF;
              float w = src[SRC32_W];
              float term = fc * fc * fl2 * w;
              acc0.add(term);
              // d/d(tx..c): term * u_k * sum_x dlog_x dG[r][x]
              float uk = a.u0h + dh;
              float dl0 = -4.f * N2[0] * fr[0] * (1.f / 0.63f),
                    dl1 = -4.f * N2[1] * fr[1] * (1.f / 0.63f),
                    dl2 = -4.f * N2[2] * fr[2] * (1.f / 0.63f);
              float tu = term * uk;
              // d term / d h_x = term dlog_x + 2 F dF/dh_x F_latt^2 w
              float fgu = 2.f * fc * fl2 * w * uk;
              float e0 = fmaf(tu, dl0, fgu * dfc[0]),
                    e1 = fmaf(tu, dl1, fgu * dfc[1]),
                    e2 = fmaf(tu, dl2, fgu * dfc[2]);
#pragma unroll
              for (int r = 0; r < 6; ++r)
                acc[r] = fmaf(e0, dG[r][0],
                              fmaf(e1, dG[r][1], fmaf(e2, dG[r][2], acc[r])));
#pragma unroll
              for (int x = 0; x < 3; ++x)
                acc[6 + x] = fmaf(term,
                                  2.f / a.N[x] -
                                      4.f * a.N[x] * fr[x] * fr[x] *
                                          (1.f / 0.63f),
                                  acc[6 + x]);
              if (HASF) {
                double gv = fscal * (double)(2.f * fc * fl2 * w);
                if (tri) {
                  if (!holding || n[0] != held[0] || n[1] != held[1] ||
                      n[2] != held[2]) {
                    flush_node();
                    held[0] = n[0];
                    held[1] = n[1];
                    held[2] = n[2];
                    holding = true;
                  }
                  // the stencil starts at fl - 1 = n - 2 + o, o = 0 or 1
                  const int o0 = fl[0] - n[0] + 1, o1 = fl[1] - n[1] + 1,
                            o2 = fl[2] - n[2] + 1;
                  const float gvf = (float)gv;
#pragma unroll
                  for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                      const float wij = gvf * (wv[0][i] * wv[1][j]);
                      const int row = ((o0 + i) * 5 + (o1 + j)) * 5 + o2;
#pragma unroll
                      for (int k = 0; k < 4; ++k)
                        s_facc[row + k][threadIdx.x] =
                            fmaf(wij, wv[2][k], s_facc[row + k][threadIdx.x]);
                    }
                } else if (inside) {
                  // consecutive terms mostly hit the same entry: add up
                  // in a register, one atomic per run of equal entries
                  if (fidx != near_idx) {
                    if (near_idx >= 0) atomicAdd(g.gradF + near_idx, near_sum);
                    near_idx = fidx;
                    near_sum = 0.0;
                  }
                  near_sum += gv;
                }
              }
            }
          }
          tot[9] += (double)scal * acc0.value();
#pragma unroll
          for (int r = 0; r < 9; ++r) tot[r] += (double)scal * (double)acc[r];
        }
#pragma unroll
    for (int r = 0; r < 9; ++r) gsum[r] = wks * tot[r];
    gsum[9] = wp * g.kc * tot[9];  // dI/dscale = I / scale
  }
  if (INTERP && HASF) flush_node();
  if (HASF && near_idx >= 0) atomicAdd(g.gradF + near_idx, near_sum);
  // block reduction in FP64, fixed order
  __shared__ double red[kTileThreads / 32][kGradN];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < kGradN; ++r) {
    double v = gsum[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][r] = v;
  }
  __syncthreads();
  if (threadIdx.x < kGradN) {
    double v = 0.0;
    for (int w = 0; w < kTileThreads / 32; ++w) v += red[w][threadIdx.x];
    g.partials[(size_t)blockIdx.x * kGradN + threadIdx.x] = v;
  }
}

// sums partial rows [n][kGradN] in a fixed order: one block of 32 x kGradN
__global__ void reduce_partials_kernel(const double *part, long long n,
                                       double *out) {
  __shared__ double red[kGradN][32];
  int r = threadIdx.y, lane = threadIdx.x;
  double v = 0.0;
  for (long long i = lane; i < n; i += 32) v += part[i * kGradN + r];
  red[r][lane] = v;
  __syncthreads();
  if (lane == 0) {
    double s = 0.0;
    for (int l = 0; l < 32; ++l) s += red[r][l];
    out[r] = s;
  }
}

// Poisson loss L = sum_p (I_p + bkg - y_p log(I_p + bkg)) and dL/dI_p
__global__ void poisson_loss_kernel(const double *img, const double *y,
                                    long long n, double bkg, double *dLdI,
                                    double *partials) {
  double l = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double m = img[i] + bkg;
    l += m - y[i] * log(m);
    dLdI[i] = 1.0 - y[i] / m;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    partials[(size_t)blockIdx.x * kGradN] = s;
  }
}

size_t adjoint_smem_bytes(const SpotArgs &a, bool f_cache) {
  return (size_t)(2 * a.PM * 9 + a.S * SRC32_STRIDE + a.PM * 54 +
                  (f_cache ? 125 * kTileThreads : 0)) *
         sizeof(float);
}

long long adjoint_blocks(const SpotArgs &a) {
  return a.pixlist ? (a.n_list + kTileThreads - 1) / kTileThreads
                   : a.n_tiles;
}

cudaError_t launch_adjoint(const SpotArgs &a, const float *dax,
                           const double *dLdI, double *gradF,
                           double *partials, double kc, double scale,
                           double *grad_out, cudaStream_t st) {
  AdjointArgs g;
  g.a = a;
  g.dax = dax;
  g.dLdI = dLdI;
  g.gradF = gradF;
  g.partials = partials;
  g.kc = kc;
  g.scale = scale;
  size_t smem = adjoint_smem_bytes(a, a.interp && gradF);
  long long blocks = adjoint_blocks(a);
  if (blocks <= 0) return cudaSuccess;
  void (*kern)(AdjointArgs) =
      a.interp ? (gradF ? spots_adjoint_kernel<1, 1> : spots_adjoint_kernel<0, 1>)
               : (gradF ? spots_adjoint_kernel<1, 0> : spots_adjoint_kernel<0, 0>);
  cudaError_t e = cudaFuncSetAttribute(
      kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)blocks, kTileThreads, smem, st>>>(g);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_partials_kernel<<<1, dim3(32, kGradN), 0, st>>>(partials, blocks,
                                                        grad_out);
  return cudaGetLastError();
}

int loss_blocks(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);
}

cudaError_t launch_poisson_loss(const double *img, const double *y,
                                long long n, double bkg, double *dLdI,
                                double *partials, double *loss_out,
                                cudaStream_t st) {
  int blocks = loss_blocks(n);
  poisson_loss_kernel<<<blocks, 256, 0, st>>>(img, y, n, bkg, dLdI, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // column 0 of the partial rows holds the block sums
  reduce_partials_kernel<<<1, dim3(32, 1), 0, st>>>(partials, blocks,
                                                   loss_out);
  return cudaGetLastError();
}

}  // namespace nbgb
