// mixed_pixel.cuh -- the per-pixel FP32-bulk Bragg-spot sum shared by the
// thread-per-pixel kernel (spots_mixed.cu) and the serving kernel
// (serve.cu).
#pragma once

#include "mixed_common.cuh"

namespace nbgb {

// Per-pixel FP32-bulk Bragg-spot sum (everything but the prefactor) of the
// pixel (s, f) of panel P, with the phi x mosaic and source tables of the
// shot staged in shared memory (s_axh/s_axl [PM][9], s_src [S][12]).  Shared
// by the thread-per-pixel kernel and the serving kernel, so that a pixel's
// value does not depend on which launch computes it.
struct PixelView {
  int PM, S;
  float u0h, u0l;
};

// Lookups of the sinc fast path: the general one (fcell_f32: tricubic, or
// nearest with its bounds test per step), and the nearest lookup with the
// index formed in FP32 and no test, for an item whose every step lands in
// the table.
enum { kLookupTable = 0, kLookupInside = 1 };

// Whether every step of an item of the sinc fast path has its nearest
// lattice point inside the table.  Along the sources h - n0 = Gq delta_q +
// rq + (a rest below ~2e-3), with delta_q in [sinc_dq[0], sinc_dq[1]] (the
// products are exact), so the step's lattice offset lies in [floor(lo),
// ceil(hi)] of the range widened by 0.01.
__device__ __forceinline__ bool sinc_item_inside(const SpotArgs &a,
                                                 const float Gq[3],
                                                 const float rq[3],
                                                 const float n0[3]) {
  bool in = true;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const float e0 = Gq[x] * a.sinc_dq[0], e1 = Gq[x] * a.sinc_dq[1];
    const float lo = floorf(fminf(e0, e1) + rq[x] - 0.01f),
                hi = ceilf(fmaxf(e0, e1) + rq[x] + 0.01f);
    const float c = n0[x] - (float)a.hmin[x];
    in = in && c + lo >= 0.f && c + hi <= (float)a.hn[x] - 1.f;
  }
  return in;
}

// h - n = sx + lo of one axis of two sources at once (the lanes), in the
// roundings of the scalar form: t = Gq dq + rq, exact (both on the 2^-21
// grid and |t| < 4), rounded to nf, sx = t - nf exact, lo = Gr delta +
// Gq dr + rr the small terms (dq, dr: delta on its grid and the rest;
// delta in FP32); returns (fh, fl) = sx + lo as a double-float pair and nf
__device__ __forceinline__ void sinc_offset2(float2 Gq, float2 Gr, float2 rq,
                                             float2 rr, float2 dq, float2 dr,
                                             float2 dd, float2 &fh, float2 &fl,
                                             float2 &nf) {
  const float2 t = ffma2(Gq, dq, rq);
  nf = make_float2(rintf(t.x), rintf(t.y));
  const float2 sx = fsub2(t, nf);
  const float2 lo = ffma2(Gr, dd, ffma2(Gq, dr, rr));
  fh = fadd2(sx, lo);
  fl = fsub2(lo, fsub2(fh, sx));
}

// One item (subpixel, phi x mosaic) of the sinc fast path over the
// sources, two at a time, added to acc in blocks of 8 sources (a plain
// FP32 sum per block).  The item's G and r are on their grids (Gq, on qG;
// rq, on 2^-21) with the rests Gr and rr; n0 is its lattice point.  q4
// holds two float4 per pair of sources 2j, 2j + 1: (dq, dq, dr, dr) and
// (w, w, delta, delta), dq = delta on the grid qD, dr the rest; a pair
// that completes an odd count has w = 0.  Gq dq is exact in FP32 (qG qD =
// 2^-21, at most 11 and 12 significant bits), and so is Gq dq + rq (on the
// 2^-21 grid, below 4 in magnitude) and its distance to the nearest n;
// the offset of the step is that value plus the small terms Gr delta +
// Gq dr + rr (|.| below ~2e-3, good to ~2e-10), kept as a double-float
// pair.  Axes h and k of one source share packed two-lane operations, and
// so do axis l, the products and the sums of the pair.
template <int INTERP, int LOOKUP>
__device__ __forceinline__ void sinc_fast_item(
    const SpotArgs &a, const float4 *q4, int S, const float Gq[3],
    const float Gr[3], const float rq[3], const float rr[3],
    const float n0[3], Kahan &acc, unsigned &evals) {
  const float hnf[3] = {(float)a.hn[0], (float)a.hn[1], (float)a.hn[2]};
  // the item's lattice point relative to the table, and its flat index
  // (integers below 2^24 in magnitude: exact in FP32)
  const float c[3] = {n0[0] - (float)a.hmin[0], n0[1] - (float)a.hmin[1],
                      n0[2] - (float)a.hmin[2]};
  const float H12 = hnf[1] * hnf[2];
  const float cidx = fmaf(c[0], H12, fmaf(c[1], hnf[2], c[2]));
  const float2 Ghk = make_float2(Gq[0], Gq[1]), Grhk = make_float2(Gr[0], Gr[1]),
               rqhk = make_float2(rq[0], rq[1]), rrhk = make_float2(rr[0], rr[1]);
  const float2 Gll = make_float2(Gq[2], Gq[2]), Grll = make_float2(Gr[2], Gr[2]),
               rqll = make_float2(rq[2], rq[2]), rrll = make_float2(rr[2], rr[2]);
  const float2 Nhk = make_float2(a.N[0], a.N[1]),
               Nll = make_float2(a.N[2], a.N[2]);
  const int P = (S + 1) >> 1;  // pairs
  for (int j0 = 0; j0 < P; j0 += 4) {
    const int jend = min(j0 + 4, P);
    float2 blk = make_float2(0.f, 0.f);
    for (int j = j0; j < jend; ++j) {
      const float4 D = q4[2 * j], Wp = q4[2 * j + 1];
      // fh[s], fl[s]: (h, k) of source s; fhl, fll: l of both sources
      float2 fh[2], fl[2], nf[2], fhl, fll, nfl;
      sinc_offset2(Ghk, Grhk, rqhk, rrhk, make_float2(D.x, D.x),
                   make_float2(D.z, D.z), make_float2(Wp.z, Wp.z), fh[0],
                   fl[0], nf[0]);
      sinc_offset2(Ghk, Grhk, rqhk, rrhk, make_float2(D.y, D.y),
                   make_float2(D.w, D.w), make_float2(Wp.w, Wp.w), fh[1],
                   fl[1], nf[1]);
      sinc_offset2(Gll, Grll, rqll, rrll, make_float2(D.x, D.y),
                   make_float2(D.z, D.w), make_float2(Wp.z, Wp.w), fhl, fll,
                   nfl);
      // nf was rounded from the grid values, which differ from h by up to
      // |lo|: h's nearest lattice point is n0 + nf plus the rounding of the
      // offset (-+1 beyond 1/2), as the table lookup needs (the sinc ratio
      // is the same for f and f -+ 1 up to its sign; the tricubic cell
      // coordinates move with it).  m: that lattice point relative to n0;
      // the lookup without bounds tests forms it only in the rare pair with
      // an offset beyond 1/2
      float m[2][3], fr[2][3];
      const bool beyond =
          LOOKUP != kLookupInside ||
          fmaxf(fmaxf(fmaxf(fabsf(fh[0].x), fabsf(fh[0].y)),
                      fmaxf(fabsf(fh[1].x), fabsf(fh[1].y))),
                fmaxf(fabsf(fhl.x), fabsf(fhl.y))) > 0.5f;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float fx[3] = {q ? fh[1].x : fh[0].x, q ? fh[1].y : fh[0].y,
                             q ? fhl.y : fhl.x};
        const float nx[3] = {q ? nf[1].x : nf[0].x, q ? nf[1].y : nf[0].y,
                             q ? nfl.y : nfl.x};
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          m[q][x] = nx[x];
          fr[q][x] = fx[x];
        }
        if (beyond) {
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            const float adj = rintf(fx[x]);
            if (INTERP == 1) fr[q][x] = __fsub_rn(fx[x], adj);
            m[q][x] = nx[x] + adj;
          }
        }
      }
      // numerators sin(pi N f) and denominators sin(pi f): (h, k) of each
      // source, l of both; their products per source in (x, y)
      const float2 nh0 = sinpi_reduced2_d4(sinc_arg2(Nhk, fh[0], fl[0]));
      const float2 nh1 = sinpi_reduced2_d4(sinc_arg2(Nhk, fh[1], fl[1]));
      const float2 nl = sinpi_reduced2_d4(sinc_arg2(Nll, fhl, fll));
      const float2 dh0 = sinpi_reduced2_d4(fh[0]);
      const float2 dh1 = sinpi_reduced2_d4(fh[1]);
      const float2 dl = sinpi_reduced2_d4(fhl);
      float2 num = fmul2(make_float2(nh0.x * nh0.y, nh1.x * nh1.y), nl);
      float2 den = fmul2(make_float2(dh0.x * dh0.y, dh1.x * dh1.y), dl);
      if (den.x == 0.f || den.y == 0.f) {
        // an offset exactly 0: that axis's ratio is N (f -> 0)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float2 fq = q ? fh[1] : fh[0], nq = q ? nh1 : nh0,
                       dq = q ? dh1 : dh0;
          const float fz = q ? fhl.y : fhl.x, nz = q ? nl.y : nl.x,
                      dz = q ? dl.y : dl.x;
          const bool z0 = fq.x == 0.f, z1 = fq.y == 0.f, z2 = fz == 0.f;
          const float nu = (z0 ? a.N[0] : nq.x) * (z1 ? a.N[1] : nq.y) *
                           (z2 ? a.N[2] : nz);
          const float de = (z0 ? 1.f : dq.x) * (z1 ? 1.f : dq.y) *
                           (z2 ? 1.f : dz);
          if (q) {
            num.y = nu;
            den.y = de;
          } else {
            num.x = nu;
            den.x = de;
          }
        }
      }
      const float2 ratio = make_float2(__fdividef(num.x, den.x),
                                       __fdividef(num.y, den.y));
      float fc[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (LOOKUP == kLookupInside) {
          const float idx =
              fmaf(m[q][0], H12, fmaf(m[q][1], hnf[2], m[q][2] + cidx));
          fc[q] = __ldg(a.F + nb_idx(a.check, NB_SITE_F, (long long)idx,
                                     table_size(a)));
        } else {
          const int n[3] = {__float2int_rn(c[0] + m[q][0]),
                            __float2int_rn(c[1] + m[q][1]),
                            __float2int_rn(c[2] + m[q][2])};
          fc[q] = fcell_f32<INTERP>(a, n, fr[q]);
        }
      }
      const float2 f2 = make_float2(fc[0], fc[1]);
      blk = ffma2(fmul2(fmul2(f2, f2), fmul2(ratio, ratio)),
                  make_float2(Wp.x, Wp.y), blk);
    }
    acc.add(blk.x + blk.y);
  }
  evals += S;
}

// s_srcq: the sinc fast path's source table in shared memory (two float4
// per pair of sources, as sinc_fast_item reads it), or null.
template <int SHAPE, int INTERP, int MODE, int HASDIV>
__device__ __forceinline__ double mixed_pixel(const SpotArgs &a,
                                              const PixelView &v,
                                              const float *s_axh,
                                              const float *s_axl,
                                              const float *s_src,
                                              const DevPanel &P, int s, int f,
                                              unsigned &evals,
                                              const float *s_srcq = nullptr) {
  const double px = P.px;
  const int os = a.os;
  const float kahn = a.kahn;
  const float cutg = kGaussCut * 0.63f;
  float th = 0.f, tl = 0.f;  // the pixel's sum as a double-float pair

  for (int i = 0; i < os; ++i) {
    for (int j = 0; j < os; ++j) {
      for (int t = 0; t < a.T; ++t) {
        // ---- per subpixel / layer: geometry
        float df[3], vh[3], vl[3], omega, cap = 1.f;
        if (MODE == 0) {
          unit_geometry_ff(a, P, s, f, i, j, t, vh, vl, df, omega);
        } else {
          float cf = (f + (i + 0.5f) / os) * (float)px,
                cs = (s + (j + 0.5f) / os) * (float)px, cn = t * a.dtff[0];
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
          float nd = pos[0] * P.ffn[0][0] + pos[1] * P.ffn[1][0] +
                     pos[2] * P.ffn[2][0];
          omega = (float)px * (float)px * nd / (R * R * R);
        }
        if (a.dtff[0] > 0.f) {
          float rho = df[0] * P.ffn[0][0] + df[1] * P.ffn[1][0] +
                      df[2] * P.ffn[2][0];
          float L = a.attenf * rho, dtf = a.dtff[0];
          cap = expf(-t * dtf / L) - expf(-(t + 1) * dtf / L);
        }
        float scal = omega * cap;
        if (!HASDIV) {
          float c2 = df[0] * a.i0ff[0][0] + df[1] * a.i0ff[1][0] +
                     df[2] * a.i0ff[2][0];
          float x = df[0] * a.e0f[0] + df[1] * a.e0f[1] +
                    df[2] * a.e0f[2];
          float y = df[0] * a.b0f[0] + df[1] * a.b0f[1] +
                    df[2] * a.b0f[2];
          scal *= 0.5f * (1.f + c2 * c2 - kahn * (x * x - y * y));
        }
        Kahan acc;
        for (int pm = 0; pm < v.PM; ++pm) {
          // ---- per (subpixel, phi x mosaic): G = A.(d - i0), r = u0 G - n0
          const float *Ah = s_axh + pm * 9, *Al = s_axl + pm * 9;
          float Gh[3], Gl[3], rh[3], rl[3], n0[3];
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            if (MODE == 0) {
              ff_dot3(Ah + 3 * x, Al + 3 * x, vh, vl, Gh[x], Gl[x]);
              float qh, qe;
              two_prod(Gh[x], v.u0h, qh, qe);
              float ql = fmaf(Gh[x], v.u0l, fmaf(Gl[x], v.u0h, qe));
              n0[x] = rintf(qh);
              two_sum(__fsub_rn(qh, n0[x]), ql, rh[x], rl[x]);
              if (SHAPE == 1) {
                // r_hi on a 2^-21 grid: r_hi - n is then exact for |n| < 7
                float rq = __fmul_rn(rintf(__fmul_rn(rh[x], 2097152.f)),
                                     1.f / 2097152.f);
                rl[x] = rl[x] + __fsub_rn(rh[x], rq);
                rh[x] = rq;
              }
            } else {
              Gh[x] = Ah[3 * x] * vh[0] + Ah[3 * x + 1] * vh[1] +
                      Ah[3 * x + 2] * vh[2];
              Gl[x] = 0.f;
              rh[x] = rl[x] = n0[x] = 0.f;
            }
          }
          // sinc in NB_MIXED, fast path (sinc_fast_item): G rounded to the
          // grid qG, r to the grid 2^-21.  Taken per item when every axis
          // has |G| < 2^11 qG and |G| max|dq| <= 3, otherwise the general
          // path below.
          bool fastq = false;
          float Gq[3], Gr[3], rq2[3], rr2[3];
          if (MODE == 0 && SHAPE == 0 && !HASDIV && s_srcq) {
            const float qG = a.sinc_qG, iqG = 1.f / qG;  // powers of 2
            // |G| < 2^11 qG keeps Gq dq exact; |G dq| <= 3 keeps
            // Gq dq + rq below 4, where the 2^-21 grid is exact in FP32
            const float dqmax =
                fmaxf(fabsf(a.sinc_dq[0]), fabsf(a.sinc_dq[1]));
            fastq = true;
#pragma unroll
            for (int x = 0; x < 3; ++x) {
              fastq = fastq && fabsf(Gh[x]) < 2048.f * qG &&
                      fabsf(Gh[x]) * dqmax <= 3.f;
              Gq[x] = __fmul_rn(rintf(__fmul_rn(Gh[x], iqG)), qG);
              Gr[x] = __fsub_rn(Gh[x], Gq[x]) + Gl[x];
              rq2[x] = __fmul_rn(rintf(__fmul_rn(rh[x], 2097152.f)),
                                 1.f / 2097152.f);
              rr2[x] = __fsub_rn(rh[x], rq2[x]) + rl[x];
            }
          }
          if (fastq) {
            const float4 *q4 = reinterpret_cast<const float4 *>(s_srcq);
            // the nearest lookup's index in FP32 for an item whose steps all
            // land in the table: a table below 2^23 entries with hn_h >= 16
            // keeps every partial sum of the index below 2^24
            if (INTERP == 0 && table_size(a) <= (1ll << 23) && a.hn[0] >= 16 &&
                sinc_item_inside(a, Gq, rq2, n0))
              sinc_fast_item<INTERP, kLookupInside>(a, q4, v.S, Gq, Gr, rq2,
                                                    rr2, n0, acc, evals);
            else
              sinc_fast_item<INTERP, kLookupTable>(a, q4, v.S, Gq, Gr, rq2,
                                                   rr2, n0, acc, evals);
            continue;
          }
          if (MODE == 0 && SHAPE == 0 && !HASDIV) {
            // sinc in NB_MIXED: the h and k axes in packed two-lane FP32
            // arithmetic, l in scalar; the numerator and denominator sines
            // of an axis pair in one packed polynomial each
            const float2 Gh2 = make_float2(Gh[0], Gh[1]),
                         Gl2 = make_float2(Gl[0], Gl[1]),
                         rh2 = make_float2(rh[0], rh[1]),
                         rl2 = make_float2(rl[0], rl[1]),
                         N2 = make_float2(a.N[0], a.N[1]);
            for (int k = 0; k < v.S; ++k) {
              const float *src = s_src + k * SRC32_STRIDE;
              const float dh = src[SRC32_DH], dl = src[SRC32_DL];
              float2 fh2, fl2v, nf2;
              frac_ff2(Gh2, Gl2, rh2, rl2, dh, dl, fh2, fl2v, nf2);
              float frz, frlz, nfz;
              frac_ff<0>(Gh[2], Gl[2], rh[2], rl[2], dh, dl, 0.f, 0.f, frz,
                         frlz, nfz);
              const float fr[3] = {fh2.x, fh2.y, frz};
              int n[3];
              n[0] = __float2int_rn(n0[0] + nf2.x) - a.hmin[0];
              n[1] = __float2int_rn(n0[1] + nf2.y) - a.hmin[1];
              n[2] = __float2int_rn(n0[2] + nfz) - a.hmin[2];
              const float2 yr2 = sinc_arg2(N2, fh2, fl2v);
              const float2 nh = sinpi_reduced2(yr2);  // numerators h, k
              const float2 dk = sinpi_reduced2(fh2);  // denominators h, k
              float yzh, yze;
              two_prod(a.N[2], frz, yzh, yze);
              const float yzl = fmaf(a.N[2], frlz, yze);
              const float yzr = __fsub_rn(yzh, rintf(yzh)) + yzl;
              const float2 sl = sinpi_reduced2(make_float2(yzr, frz));
              // at a lattice point (|f| < 1e-9) the ratio is N
              const bool z0 = fabsf(fh2.x) < 1e-9f, z1 = fabsf(fh2.y) < 1e-9f,
                         z2 = fabsf(frz) < 1e-9f;
              const float num = (z0 ? a.N[0] : nh.x) * (z1 ? a.N[1] : nh.y) *
                                (z2 ? a.N[2] : sl.x);
              const float den = (z0 ? 1.f : dk.x) * (z1 ? 1.f : dk.y) *
                                (z2 ? 1.f : sl.y);
              const float ratio = __fdividef(num, den);
              ++evals;
              const float fc = fcell_f32<INTERP>(a, n, fr);
              acc.add(fc * fc * (ratio * ratio) * src[SRC32_W]);
            }
            continue;
          }
          for (int k = 0; k < v.S; ++k) {
            const float *src = s_src + k * SRC32_STRIDE;
            float fr[3], frl[3];
            int n[3];
#pragma unroll
            for (int x = 0; x < 3; ++x) {
              float Eh = 0.f, El = 0.f;
              if (HASDIV) {
                size_t e = ((size_t)pm * v.S + k) * 3 + x;
                Eh = __ldg(a.divh + e);
                El = __ldg(a.divl + e);
              }
              float nf;
              if (MODE == 0 && SHAPE == 1) {
                // Gaussian: cheap offset for the cut test, refined below
                float t = fmaf(Gh[x], src[SRC32_DH], rh[x]);
                nf = rintf(t);
                fr[x] = t - nf;
                frl[x] = nf;  // keeps the shift for the refinement
                if (HASDIV) {
                  fr[x] -= Eh;
                  float n2 = rintf(fr[x]);
                  fr[x] -= n2;
                  nf += n2;
                }
              } else if (MODE == 0) {
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
              if (MODE == 0) {
                // precise offset: G_hi d_hi + (r_q - n) in one rounding plus
                // the small terms (and the divergence term, re-centred)
#pragma unroll
                for (int x = 0; x < 3; ++x) {
                  float nfx = frl[x];
                  float sx = fmaf(Gh[x], src[SRC32_DH], __fsub_rn(rh[x], nfx));
                  float c = fmaf(Gh[x], src[SRC32_DL],
                                 fmaf(Gl[x], src[SRC32_DH], rl[x]));
                  fr[x] = sx + c;
                  if (HASDIV) {
                    // h - n0 - nfx - E, re-centred; the index follows it
                    size_t e = ((size_t)pm * v.S + k) * 3 + x;
                    fr[x] -= __ldg(a.divh + e) + __ldg(a.divl + e);
                    float n2 = rintf(fr[x]);
                    fr[x] -= n2;
                    n[x] = __float2int_rn(n0[x] + nfx + n2) - a.hmin[x];
                  }
                }
                rad2 = a.N[0] * a.N[0] * fr[0] * fr[0];
                rad2 = fmaf(a.N[1] * a.N[1], fr[1] * fr[1], rad2);
                rad2 = fmaf(a.N[2] * a.N[2], fr[2] * fr[2], rad2);
              }
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
        // the unit's compensated sum times scal, added in double-float
        {
          float uh, ul, ph, pl;
          fast_two_sum(acc.s, -acc.c, uh, ul);
          ff_mul(uh, ul, scal, 0.f, ph, pl);
          ff_add(th, tl, ph, pl, th, tl);
        }
      }
    }
  }
  return (double)th + (double)tl;
}

}  // namespace nbgb
