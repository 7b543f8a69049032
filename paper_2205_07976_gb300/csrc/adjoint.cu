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
  // term-ring kernel: rows of 32 pixels handed to warps by a counter;
  // partials holds one row of the ten sums per pixel row
  unsigned long long *rows_next;
  long long n_rows;
};

constexpr int kGradN = 10;

// Value F and gradient (dF/dx, dF/dy, dF/dz) at x in [0, 1)^3 of a cell's
// tricubic polynomial, its 64 monomial coefficients C[a][b][c] of
// x^a y^b z^c at cp in the layout of SpotArgs::C4: nested Horner in z, y,
// x carrying the derivatives along, the chains of x^(2P) and x^(2P+1)
// side by side in packed two-lane FMAs.
__device__ __forceinline__ void cell_value_grad(const float4 *cp,
                                                const float x[3], float &F,
                                                float dF[3]) {
  const float2 z2 = make_float2(x[2], x[2]), y2 = make_float2(x[1], x[1]);
  float2 q[2], qy[2], qz[2];
#pragma unroll
  for (int P = 0; P < 2; ++P) {
    float2 pb[4], db[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float4 A = __ldg(cp + (P * 4 + b) * 2);
      const float4 B = __ldg(cp + (P * 4 + b) * 2 + 1);
      // p = ((c3 z + c2) z + c1) z + c0 and its z-derivative
      float2 p = make_float2(A.x, A.y);
      float2 d = p;
      p = ffma2(p, z2, make_float2(A.z, A.w));
      d = ffma2(d, z2, p);
      p = ffma2(p, z2, make_float2(B.x, B.y));
      d = ffma2(d, z2, p);
      p = ffma2(p, z2, make_float2(B.z, B.w));
      pb[b] = p;
      db[b] = d;
    }
    // Horner in y over b = 3 .. 0: value, y-derivative, z-derivative
    float2 v = pb[3], vy = pb[3], vz = db[3];
    v = ffma2(v, y2, pb[2]);
    vz = ffma2(vz, y2, db[2]);
    vy = ffma2(vy, y2, v);
    v = ffma2(v, y2, pb[1]);
    vz = ffma2(vz, y2, db[1]);
    vy = ffma2(vy, y2, v);
    v = ffma2(v, y2, pb[0]);
    vz = ffma2(vz, y2, db[0]);
    q[P] = v;
    qy[P] = vy;
    qz[P] = vz;
  }
  // q[P] = (Q_{2P}, Q_{2P+1}); Horner in x over a = 3 .. 0
  const float xx = x[0];
  float v = q[1].y, vx = q[1].y, vy = qy[1].y, vz = qz[1].y;
  v = fmaf(v, xx, q[1].x);
  vy = fmaf(vy, xx, qy[1].x);
  vz = fmaf(vz, xx, qz[1].x);
  vx = fmaf(vx, xx, v);
  v = fmaf(v, xx, q[0].y);
  vy = fmaf(vy, xx, qy[0].y);
  vz = fmaf(vz, xx, qz[0].y);
  vx = fmaf(vx, xx, v);
  v = fmaf(v, xx, q[0].x);
  vy = fmaf(vy, xx, qy[0].x);
  vz = fmaf(vz, xx, qz[0].x);
  F = v;
  dF[0] = vx;
  dF[1] = vy;
  dF[2] = vz;
}

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
  extern __shared__ __align__(16) float smf[];
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
  // its run of terms, summed in FP32 (an FP64 instruction per term would
  // cost 64 FP32 ones on this part) and added to the FP64 gradient once
  float near_sum = 0.f;
  int held[3] = {0, 0, 0};  // the lattice point held (table-relative)
  bool holding = false;
  auto flush_node = [&]() {
    if (!holding) return;
    for (int e = 0; e < 125; ++e) {
      const float v = s_facc[e][threadIdx.x];
      if (v == 0.f) continue;  // untouched (may lie outside the table)
      s_facc[e][threadIdx.x] = 0.f;
      const int i = e / 25, j = (e / 5) % 5, k = e % 5;
      atomicAdd(g.gradF + nb_idx(a.check, NB_SITE_GRADF,
                                 ((long long)(held[0] - 2 + i) * a.hn[1] +
                                  (held[1] - 2 + j)) * a.hn[2] +
                                     (held[2] - 2 + k),
                                 table_size(a)),
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
          const float fscal = (float)(wks * (double)scal);  // F scatter
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
                      const float *row = a.F + stencil_row(a, fl, i, j);
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
              if (!tri) fc = inside ? __ldg(a.F + nb_idx(a.check, NB_SITE_F, fidx, table_size(a))) : a.defF;
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
                const float gvf = fscal * (2.f * fc * fl2 * w);
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
                    if (near_idx >= 0) atomicAdd(g.gradF + nb_idx(a.check, NB_SITE_GRADF, near_idx, table_size(a)), (double)near_sum);
                    near_idx = fidx;
                    near_sum = 0.f;
                  }
                  near_sum += gvf;
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
  if (HASF && near_idx >= 0) atomicAdd(g.gradF + nb_idx(a.check, NB_SITE_GRADF, near_idx, table_size(a)), (double)near_sum);
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

// ---------------------------------------------------------------------
// Term-ring form (used where every table axis is at most 1000 long).  The
// thread-per-pixel kernel above evaluates a surviving term in the lane of
// its pixel, so a warp runs its expensive tricubic terms (64 table reads
// for the value, gradient and weights, 64 column updates) with only the
// lanes whose pixel has a term at that step.  Here the lanes still scan
// their own pixels' steps in lockstep (every pixel has the same steps),
// but a surviving step is pushed as a record into a per-warp ring in
// shared memory, and whenever the ring holds 32 records the warp
// evaluates them one per lane.  A record carries the step's exact offset,
// its lattice point, its (phi x mosaic, source) indices and the lane of
// its pixel, whose unit geometry and weight dL/dI K cap pol omega sit in a
// per-warp table.  Each lane adds what it evaluates into FP32 sums, which
// the warp folds into FP64 every 16 passes with a fixed butterfly, so the
// ten scalars stay deterministic.
constexpr int kAdjRing = 64;  // pending < 32 after a pass, + 32 pushed
constexpr int kAdjFold = 16;  // passes between folds into FP64

__host__ __device__ inline size_t adj_ring_floats(int PM, int S,
                                                  bool f_cache) {
  // the tables, then (F gradient) each thread's 5x5x4 column as 25 float4
  // (16-byte aligned: 2 PM 9 + 12 S + 54 PM is a multiple of 4)
  size_t fl = (size_t)2 * PM * 9 + (size_t)S * SRC32_STRIDE + (size_t)PM * 54 +
              (f_cache ? (size_t)100 * kTileThreads : 0);
  return (fl + 3) & ~(size_t)3;  // 16-byte aligned records after it
}

__host__ __device__ inline size_t adj_ring_smem_bytes(int PM, int S,
                                                      bool f_cache) {
  const int warps = kTileThreads / 32;
  return adj_ring_floats(PM, S, f_cache) * sizeof(float) +
         (size_t)warps * kAdjRing * (sizeof(float4) + sizeof(int)) +
         (size_t)warps * 32 * (sizeof(float4) + sizeof(int));
}

template <int HASF, int INTERP>
__global__ void __launch_bounds__(kTileThreads, INTERP ? 3 : 4)
    spots_adjoint_ring_kernel(AdjointArgs g) {
  const SpotArgs &a = g.a;
  extern __shared__ __align__(16) float smf[];
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
  const bool fcache = INTERP && HASF;
  float4 (*s_col)[kTileThreads] =
      reinterpret_cast<float4 (*)[kTileThreads]>(s_dax + a.PM * 54);
  float4 *s_rec = reinterpret_cast<float4 *>(
      smf + adj_ring_floats(a.PM, a.S, fcache));
  int *s_recb = reinterpret_cast<int *>(s_rec + (kTileThreads / 32) * kAdjRing);
  float4 *s_unit =
      reinterpret_cast<float4 *>(s_recb + (kTileThreads / 32) * kAdjRing);
  int *s_perm = reinterpret_cast<int *>(s_unit + (kTileThreads / 32) * 32);
  if (fcache)
    for (int r = 0; r < 25; ++r)
      s_col[r][threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4 *rec_a = s_rec + warp * kAdjRing;
  int *rec_b = s_recb + warp * kAdjRing;
  float4 *unit_w = s_unit + warp * 32;
  int *perm = s_perm + warp * 32;

  // structure-factor gradient state of this lane.  A tricubic term near
  // lattice point n with its cell starting at fl touches nodes
  // fl - 1 .. fl + 2 on each axis: the lane sums them in a column of 5 x 5
  // nodes around (n_h, n_k) by the 4 nodes fl_l - 1 .. fl_l + 2 along l (a
  // float4 per (h, k) node), keyed by (n_h, n_k, fl_l) packed like a
  // record's lattice point (-1: no column)
  long long near_idx = -1;
  double near_sum = 0.0;
  int held_key = -1;
  // Flushes, cooperatively, the columns of the lanes with `need`: lanes
  // with the same key are summed entry by entry (in FP32, in lane order)
  // and each touched node gets one FP64 atomic; the 100 entries of a group
  // are split over the 32 lanes.  Called by all lanes.
  auto flush_columns = [&](bool need) {
    unsigned todo = __ballot_sync(0xffffffffu, need && held_key >= 0);
    while (todo) {
      const int key = __shfl_sync(0xffffffffu, held_key, __ffs(todo) - 1);
      const unsigned grp =
          __ballot_sync(0xffffffffu, need && held_key == key && key >= 0);
      todo &= ~grp;
      const int c0 = (key & 1023) - 1, c1 = ((key >> 10) & 1023) - 1,
                c2 = ((key >> 20) & 1023) - 1;
      for (int e = lane; e < 100; e += 32) {
        const int r = e >> 2, kk = e & 3;
        float v = 0.f;
        for (unsigned m = grp; m; m &= m - 1) {
          float *col = reinterpret_cast<float *>(
              &s_col[r][warp * 32 + __ffs(m) - 1]);
          v += col[kk];
          col[kk] = 0.f;
        }
        if (v != 0.f)
          atomicAdd(g.gradF + nb_idx(a.check, NB_SITE_GRADF,
                                     ((long long)(c0 - 2 + r / 5) * a.hn[1] +
                                      (c1 - 2 + r % 5)) * a.hn[2] +
                                         (c2 - 1 + kk),
                                     table_size(a)),
                    (double)v);
      }
    }
    if (need) held_key = -1;
    __syncwarp();
  };
  // a record's column key: its lattice point with l replaced by the start
  // of its cell along l
  auto column_key = [&](float4 ra) {
    const int npk = __float_as_int(ra.w);
    return (npk & 0xfffff) |
           ((((npk >> 20) & 1023) - (ra.z < 0.f ? 1 : 0)) << 20);
  };

  const float N2[3] = {a.N[0] * a.N[0], a.N[1] * a.N[1], a.N[2] * a.N[2]};
  const float cutg = kGaussCut * 0.63f;
  const float kahn = a.kahn;
  const float scalef = (float)g.scale;

  float acc[kGradN];
#pragma unroll
  for (int r = 0; r < kGradN; ++r) acc[r] = 0.f;
  double dacc = 0.0;  // lane r < kGradN: the warp's folded sum r
  int head = 0, tail = 0, passes = 0;

  auto fold = [&]() {
#pragma unroll
    for (int r = 0; r < kGradN; ++r) {
      float v = acc[r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == r) dacc += (double)v;
      acc[r] = 0.f;
    }
  };
  // evaluates records head .. head + cnt - 1 (cnt <= 32), one per lane
  auto eval_pass = [&](int cnt) {
    const bool v = lane < cnt;
    int slot = (head + lane) & (kAdjRing - 1);
    if (HASF) {
      // the pass's records in the order of their lattice points (ties in
      // ring order): lanes then keep the node of their column across
      // passes more often, and flush it less
      const int key = v ? column_key(rec_a[slot]) : 0x7fffffff;
      bool placed = !v;
      int pos = 0, base = 0;
      while (__any_sync(0xffffffffu, !placed)) {
        const int kmin = __reduce_min_sync(0xffffffffu, placed ? 0x7fffffff : key);
        const unsigned grp = __ballot_sync(0xffffffffu, !placed && key == kmin);
        if (!placed && key == kmin) {
          pos = base + __popc(grp & ((1u << lane) - 1u));
          placed = true;
        }
        base += __popc(grp);
      }
      if (v) perm[pos] = slot;
      __syncwarp();
      if (v) slot = perm[lane];
      __syncwarp();
      // a lane whose record has another column key than its column
      // flushes the column first
      if (INTERP)
        flush_columns(v && held_key >= 0 &&
                      column_key(rec_a[slot]) != held_key);
    }
    head += cnt;
    if (v) {
      const float4 ra = rec_a[slot];
      const int rb = rec_b[slot];
      const float fr[3] = {ra.x, ra.y, ra.z};
      const int npk = __float_as_int(ra.w);
      int n[3];
#pragma unroll
      for (int x = 0; x < 3; ++x) n[x] = ((npk >> (10 * x)) & 1023) - 1;
      const int pm = rb & 2047, k = (rb >> 11) & 1023, sl = (rb >> 21) & 31;
      const float4 uw = unit_w[sl];
      const float v32[3] = {uw.x, uw.y, uw.z};
      const float Wt = uw.w;
      const float *src = s_src + k * SRC32_STRIDE;
      const float dh = src[SRC32_DH], w = src[SRC32_W];
      float rad2 = N2[0] * fr[0] * fr[0];
      rad2 = fmaf(N2[1] * fr[1], fr[1], rad2);
      rad2 = fmaf(N2[2] * fr[2], fr[2], rad2);
      const float fl2 = a.N6 * expf(-2.f * rad2 * (1.f / 0.63f));
      const bool inside = (unsigned)n[0] < (unsigned)a.hn[0] &&
                          (unsigned)n[1] < (unsigned)a.hn[1] &&
                          (unsigned)n[2] < (unsigned)a.hn[2];
      const long long fidx =
          inside ? ((long long)n[0] * a.hn[1] + n[1]) * a.hn[2] + n[2] : -1;
      float fc, dfc[3] = {0.f, 0.f, 0.f};
      bool tri = false;
      int fl[3];
      float wv[3][4];
      if (INTERP == 1) {
        float xs[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int neg = fr[c] < 0.f;
          fl[c] = n[c] - neg;
          xs[c] = neg ? 1.f + fr[c] : fr[c];
        }
        tri = fl[0] >= 1 && fl[0] + 2 < a.hn[0] && fl[1] >= 1 &&
              fl[1] + 2 < a.hn[1] && fl[2] >= 1 && fl[2] + 2 < a.hn[2];
        if (tri && a.C4) {
          // value and gradient of the cell's polynomial (its 64 monomial
          // coefficients), and the Lagrange weights for the F scatter
#pragma unroll
          for (int c = 0; c < 3; ++c) lagrange4(xs[c], wv[c]);
          const int ci = ((fl[0] - 1) * (a.hn[1] - 3) + (fl[1] - 1)) *
                             (a.hn[2] - 3) +
                         (fl[2] - 1);
          cell_value_grad(
              a.C4 + (size_t)nb_idx(a.check, NB_SITE_CELL, ci, cell_count(a)) * 16,
              xs, fc, dfc);
        } else if (tri) {
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
                  a.F + stencil_row(a, fl, i, j);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const float Fv = __ldg(row + kk);
                const float wij = wv[0][i] * wv[1][j];
                fc = fmaf(wij * wv[2][kk], Fv, fc);
                dfc[0] = fmaf(wd[0][i] * wv[1][j] * wv[2][kk], Fv, dfc[0]);
                dfc[1] = fmaf(wv[0][i] * wd[1][j] * wv[2][kk], Fv, dfc[1]);
                dfc[2] = fmaf(wij * wd[2][kk], Fv, dfc[2]);
              }
            }
        }
      }
      if (!tri) fc = inside ? __ldg(a.F + nb_idx(a.check, NB_SITE_F, fidx, table_size(a))) : a.defF;
      const float term = fc * fc * fl2 * w;
      const float uk = a.u0h + dh;
      const float tu = term * uk, fgu = 2.f * fc * fl2 * w * uk;
      float e[3];
#pragma unroll
      for (int x = 0; x < 3; ++x)
        e[x] = fmaf(tu, -4.f * N2[x] * fr[x] * (1.f / 0.63f), fgu * dfc[x]);
      // d term / d theta_r = sum_x e_x dA_pm[r][x] . v
      const float *dA = s_dax + pm * 54;
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        float gr = 0.f;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          const float *d3 = dA + r * 9 + 3 * x;
          gr = fmaf(e[x], d3[0] * v32[0] + d3[1] * v32[1] + d3[2] * v32[2],
                    gr);
        }
        acc[r] = fmaf(Wt, gr, acc[r]);
      }
      const float tw = Wt * term;
#pragma unroll
      for (int x = 0; x < 3; ++x)
        acc[6 + x] = fmaf(tw, 2.f / a.N[x] - 4.f * a.N[x] * fr[x] * fr[x] *
                                                 (1.f / 0.63f),
                          acc[6 + x]);
      acc[9] += tw;
      if (HASF) {
        const float gvf = Wt * scalef * (2.f * fc * fl2 * w);
        if (tri) {
          // the column was flushed unless it holds this key
          held_key = (npk & 0xfffff) | ((fl[2] + 1) << 20);
          const int o0 = fl[0] - n[0] + 1, o1 = fl[1] - n[1] + 1;
          float4 *col = &s_col[o0 * 5 + o1][threadIdx.x];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const float wij = gvf * (wv[0][i] * wv[1][j]);
              float4 c = col[(i * 5 + j) * kTileThreads];
              c.x = fmaf(wij, wv[2][0], c.x);
              c.y = fmaf(wij, wv[2][1], c.y);
              c.z = fmaf(wij, wv[2][2], c.z);
              c.w = fmaf(wij, wv[2][3], c.w);
              col[(i * 5 + j) * kTileThreads] = c;
            }
        } else if (inside) {
          if (fidx != near_idx) {
            if (near_idx >= 0) atomicAdd(g.gradF + nb_idx(a.check, NB_SITE_GRADF, near_idx, table_size(a)), near_sum);
            near_idx = fidx;
            near_sum = 0.0;
          }
          near_sum += (double)gvf;
        }
      }
    }
    __syncwarp();
    if (++passes % kAdjFold == 0) fold();
  };

  // Each warp takes rows of 32 pixels (a warp's quarter of a 16x8 tile, or
  // 32 entries of the pixel list) from a counter, and per pixel its steps
  // (unit, phi x mosaic, source): one step per iteration, the same
  // sequence in every lane.  The ring is drained before a unit's row of
  // the unit table is rewritten and at the end of a pixel row, whose ten
  // sums then go to the row's own partial row: the sums do not depend on
  // which warp took which row.
  const int U = a.os * a.os * a.T;
  auto next_row = [&]() {
    unsigned long long r = 0;
    if (lane == 0) r = atomicAdd(g.rows_next, 1ull);
    return (long long)__shfl_sync(0xffffffffu, r, 0);
  };
  long long row = next_row();
  bool row_done = false;
  int u = 0, pm = 0, k = 0;
  bool new_pixel = true, new_unit = true, new_pm = true;
  bool ok = false;
  const DevPanel *P = a.panels;
  int s = 0, f = 0;
  float W0 = 0.f;
  float vh[3], vl[3];
  float Gh[3], Gl[3], rq[3], rl[3], n0[3];
  while (true) {
    const bool finished = row >= g.n_rows;
    if (tail - head >= 32 ||
        ((finished || new_unit || row_done) && tail > head)) {
      eval_pass(min(32, tail - head));
      continue;
    }
    if (row_done) {
      // the row's records are all evaluated: its sums, then the next row
      fold();
      if (lane < kGradN)
        g.partials[(size_t)row * kGradN + lane] =
            lane < 9 ? g.scale * dacc : dacc;
      dacc = 0.0;
      passes = 0;
      row = next_row();
      row_done = false;
      new_pixel = new_unit = new_pm = true;
      continue;
    }
    if (finished) break;
    if (new_pixel) {
      long long gp = 0;
      int q = 0;
      ok = a.pixlist
               ? map_pixel(a, row * 32 + lane, lane, gp, q, s, f)
               : map_pixel(a, row / (kTileThreads / 32),
                           (int)(row % (kTileThreads / 32)) * 32 + lane, gp,
                           q, s, f);
      if (!ok) {
        q = 0;
        s = 0;
        f = 0;
      }
      P = a.panels + q;
      W0 = ok ? (float)(g.dLdI[gp] * g.kc) : 0.f;
      new_pixel = false;
    }
    if (new_unit) {
      const int t = u % a.T, ij = u / a.T, i = ij / a.os, j = ij % a.os;
      float df[3], omega;
      unit_geometry_ff(a, *P, s, f, i, j, t, vh, vl, df, omega);
      float cap = 1.f;
      if (a.dtff[0] > 0.f) {
        const float rho = df[0] * P->ffn[0][0] + df[1] * P->ffn[1][0] +
                          df[2] * P->ffn[2][0];
        const float L = a.attenf * rho, dtf = a.dtff[0];
        cap = expf(-t * dtf / L) - expf(-(t + 1) * dtf / L);
      }
      const float c2 = df[0] * a.i0ff[0][0] + df[1] * a.i0ff[1][0] +
                       df[2] * a.i0ff[2][0],
                  xe = df[0] * a.e0f[0] + df[1] * a.e0f[1] + df[2] * a.e0f[2],
                  ye = df[0] * a.b0f[0] + df[1] * a.b0f[1] + df[2] * a.b0f[2];
      const float scal = omega * cap * 0.5f *
                         (1.f + c2 * c2 - kahn * (xe * xe - ye * ye));
      unit_w[lane] = make_float4(vh[0], vh[1], vh[2], W0 * scal);
      __syncwarp();
      new_unit = false;
    }
    if (new_pm) {
      const float *Ah = s_axh + pm * 9, *Al = s_axl + pm * 9;
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        ff_dot3(Ah + 3 * x, Al + 3 * x, vh, vl, Gh[x], Gl[x]);
        float qh, qe;
        two_prod(Gh[x], a.u0h, qh, qe);
        const float ql = fmaf(Gh[x], a.u0l, fmaf(Gl[x], a.u0h, qe));
        n0[x] = rintf(qh);
        float rh, rl0;
        two_sum(__fsub_rn(qh, n0[x]), ql, rh, rl0);
        rq[x] = __fmul_rn(rintf(__fmul_rn(rh, 2097152.f)), 1.f / 2097152.f);
        rl[x] = rl0 + __fsub_rn(rh, rq[x]);
      }
      new_pm = false;
    }
    // step (u, pm, k): the cheap cut test, then the exact offset of a
    // surviving step and its record
    {
      const float *src = s_src + k * SRC32_STRIDE;
      const float dh = src[SRC32_DH], dl = src[SRC32_DL];
      float fr[3], nf[3];
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const float tq = fmaf(Gh[x], dh, rq[x]);
        nf[x] = rintf(tq);
        fr[x] = tq - nf[x];
      }
      float rad2 = N2[0] * fr[0] * fr[0];
      rad2 = fmaf(N2[1] * fr[1], fr[1], rad2);
      rad2 = fmaf(N2[2] * fr[2], fr[2], rad2);
      const bool hit = ok && rad2 <= cutg;
      const unsigned hm = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        int npk = 0;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          const float sx = fmaf(Gh[x], dh, __fsub_rn(rq[x], nf[x]));
          fr[x] = sx + fmaf(Gh[x], dl, fmaf(Gl[x], dh, rl[x]));
          const int nx = __float2int_rn(n0[x] + nf[x]) - a.hmin[x];
          npk |= (min(max(nx, -1), a.hn[x]) + 1) << (10 * x);
        }
        const int slot =
            (tail + __popc(hm & ((1u << lane) - 1u))) & (kAdjRing - 1);
        rec_a[slot] = make_float4(fr[0], fr[1], fr[2], __int_as_float(npk));
        rec_b[slot] = pm | (k << 11) | (lane << 21);
      }
      tail += __popc(hm);
      __syncwarp();
    }
    // advance (u, pm, k); after the last step of the row's pixels the row
    // is done once its records are evaluated
    if (++k == a.S) {
      k = 0;
      new_pm = true;
      if (++pm == a.PM) {
        pm = 0;
        new_unit = true;
        if (++u == U) {
          u = 0;
          row_done = true;
        }
      }
    }
  }
  if (fcache) flush_columns(true);
  if (HASF && near_idx >= 0) atomicAdd(g.gradF + nb_idx(a.check, NB_SITE_GRADF, near_idx, table_size(a)), near_sum);
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

// The term-ring kernel serves tricubic lookup (its terms are the
// expensive ones: value and gradient of the cell polynomial and 64 column
// updates); it packs a table index in 10 bits per axis.  Nearest lookup
// stays on the thread-per-pixel kernel, which measured as fast or faster.
static bool adjoint_ring_ok(const SpotArgs &a) {
  return a.interp == 1 && a.hn[0] <= 1000 && a.hn[1] <= 1000 &&
         a.hn[2] <= 1000;
}

size_t adjoint_smem_bytes(const SpotArgs &a, bool f_cache) {
  if (adjoint_ring_ok(a)) return adj_ring_smem_bytes(a.PM, a.S, f_cache);
  return (size_t)(2 * a.PM * 9 + a.S * SRC32_STRIDE + a.PM * 54 +
                  (f_cache ? 125 * kTileThreads : 0)) *
         sizeof(float);
}

// rows of partial sums the adjoint writes: one per pixel row of 32 (term
// ring) or per block (thread kernel)
long long adjoint_blocks(const SpotArgs &a) {
  if (adjoint_ring_ok(a))
    return a.pixlist ? (a.n_list + 31) / 32
                     : (long long)a.n_tiles * (kTileThreads / 32);
  return a.pixlist ? (a.n_list + kTileThreads - 1) / kTileThreads
                   : a.n_tiles;
}

cudaError_t launch_adjoint(const SpotArgs &a, const float *dax,
                           const double *dLdI, double *gradF,
                           double *partials, double kc, double scale,
                           double *grad_out, int sm_count, cudaStream_t st) {
  AdjointArgs g;
  g.a = a;
  g.dax = dax;
  g.dLdI = dLdI;
  g.gradF = gradF;
  g.partials = partials;
  g.kc = kc;
  g.scale = scale;
  g.rows_next = nullptr;
  g.n_rows = 0;
  size_t smem = adjoint_smem_bytes(a, a.interp && gradF);
  long long blocks = adjoint_blocks(a);
  if (blocks <= 0) return cudaSuccess;
  void (*kern)(AdjointArgs);
  if (adjoint_ring_ok(a))  // tricubic only
    kern = gradF ? spots_adjoint_ring_kernel<1, 1>
                 : spots_adjoint_ring_kernel<0, 1>;
  else
    kern = a.interp ? (gradF ? spots_adjoint_kernel<1, 1>
                             : spots_adjoint_kernel<0, 1>)
                    : (gradF ? spots_adjoint_kernel<1, 0>
                             : spots_adjoint_kernel<0, 0>);
  cudaError_t e = cudaFuncSetAttribute(
      kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  long long grid = blocks;
  if (adjoint_ring_ok(a)) {
    // persistent blocks; warps take pixel rows from a counter stored after
    // the partial rows (the buffer holds blocks + 1 rows)
    g.n_rows = blocks;
    g.rows_next = reinterpret_cast<unsigned long long *>(partials +
                                                        blocks * kGradN);
    e = cudaMemsetAsync(g.rows_next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern,
                                                      kTileThreads, smem);
    if (e != cudaSuccess) return e;
    const long long fit = (long long)(sm_count > 0 ? sm_count : 1) *
                          (per_sm > 0 ? per_sm : 1);
    const long long need = (blocks + kTileThreads / 32 - 1) / (kTileThreads / 32);
    grid = fit < need ? fit : need;
  }
  kern<<<(unsigned)grid, kTileThreads, smem, st>>>(g);
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
