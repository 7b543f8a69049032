// mixed_common.cuh -- device helpers shared by the FP32-bulk kernels:
// the double-float dot product, the double-float fractional offset, and
// the FP32 structure-factor lookup (nearest / tricubic).
#pragma once

#include "nbgb_internal.cuh"

namespace nbgb {

// Packed two-lane FP32 arithmetic (Blackwell's f32x2 instructions): one
// instruction rounds each lane exactly as the scalar fmaf / add / sub / mul
// does.
__device__ __forceinline__ unsigned long long pk2(float2 v) {
  return (unsigned long long)__float_as_uint(v.x) |
         ((unsigned long long)__float_as_uint(v.y) << 32);
}
__device__ __forceinline__ float2 upk2(unsigned long long v) {
  return make_float2(__uint_as_float((unsigned)v),
                     __uint_as_float((unsigned)(v >> 32)));
}
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
  return upk2(d);
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}

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

// double-float sum and product (error-free transformations + one
// renormalisation): about 48 significant bits in FP32 arithmetic
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl,
                                       float &sh, float &sl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  fast_two_sum(s, e, sh, sl);
}

__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl,
                                       float &ph, float &pl) {
  float p, e;
  two_prod(ah, bh, p, e);
  e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
  fast_two_sum(p, e, ph, pl);
}

// Geometry of sub-pixel unit (i, j, layer t) of pixel (s, f) of panel P in
// double-float FP32 arithmetic (FP64 issues at 1/64 of the FP32 rate on
// this part): v = d - i0 as (vh, vl), d rounded to FP32, and the solid
// angle omega = px^2 (n . P) / |P|^3 in FP32.  The reciprocal length is
// the FP32 rsqrt estimate refined by one Newton step carried in
// double-float, so d is good to ~1e-13.
__device__ __forceinline__ void unit_geometry_ff(const SpotArgs &a,
                                                 const DevPanel &P, int s,
                                                 int f, int i, int j, int t,
                                                 float vh[3], float vl[3],
                                                 float df[3], float &omega) {
  const float osf = (float)a.os;
  // (i + 1/2) / os and (j + 1/2) / os as double-float pairs
  const float oih = __fdiv_rn(i + 0.5f, osf);
  const float oil = __fdiv_rn(__fmaf_rn(-oih, osf, i + 0.5f), osf);
  const float ojh = __fdiv_rn(j + 0.5f, osf);
  const float ojl = __fdiv_rn(__fmaf_rn(-ojh, osf, j + 0.5f), osf);
  float uh, ul, wh, wl;
  ff_add((float)f, 0.f, oih, oil, uh, ul);  // f, s are exact in FP32
  ff_add((float)s, 0.f, ojh, ojl, wh, wl);
  float cfh, cfl, csh, csl, cnh, cnl;
  ff_mul(uh, ul, P.ffpx[0], P.ffpx[1], cfh, cfl);
  ff_mul(wh, wl, P.ffpx[0], P.ffpx[1], csh, csl);
  ff_mul((float)t, 0.f, a.dtff[0], a.dtff[1], cnh, cnl);
  float ph[3], pl[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float th, tl;
    ph[c] = P.ffo[c][0];
    pl[c] = P.ffo[c][1];
    ff_mul(cfh, cfl, P.fff[c][0], P.fff[c][1], th, tl);
    ff_add(ph[c], pl[c], th, tl, ph[c], pl[c]);
    ff_mul(csh, csl, P.ffs[c][0], P.ffs[c][1], th, tl);
    ff_add(ph[c], pl[c], th, tl, ph[c], pl[c]);
    ff_mul(cnh, cnl, P.ffn[c][0], P.ffn[c][1], th, tl);
    ff_add(ph[c], pl[c], th, tl, ph[c], pl[c]);
  }
  float r2h, r2l, th, tl;
  ff_mul(ph[0], pl[0], ph[0], pl[0], r2h, r2l);
  ff_mul(ph[1], pl[1], ph[1], pl[1], th, tl);
  ff_add(r2h, r2l, th, tl, r2h, r2l);
  ff_mul(ph[2], pl[2], ph[2], pl[2], th, tl);
  ff_add(r2h, r2l, th, tl, r2h, r2l);
  // y ~ |P|^-1; e = 1 - |P|^2 y^2 (small, 1 - qh is exact); y (1 + e/2)
  const float y = rsqrtf(r2h);
  float yy, yye, qh, ql;
  two_prod(y, y, yy, yye);
  ff_mul(r2h, r2l, yy, yye, qh, ql);
  const float e = __fsub_rn(__fsub_rn(1.f, qh), ql);
  float rih, ril;
  fast_two_sum(y, 0.5f * y * e, rih, ril);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float dh, dl;
    ff_mul(ph[c], pl[c], rih, ril, dh, dl);
    df[c] = dh;
    ff_add(dh, dl, -a.i0ff[c][0], -a.i0ff[c][1], vh[c], vl[c]);
  }
  const float nd = P.ffn[0][0] * ph[0] + P.ffn[1][0] * ph[1] +
                   P.ffn[2][0] * ph[2];
  omega = P.ffpx[0] * P.ffpx[0] * nd * (rih * rih * rih);
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

// frac_ff<0> for two axes at once (the lanes of the float2s), with the
// same roundings lane by lane; the negations are moved into the operands
// (exact in IEEE arithmetic).
__device__ __forceinline__ void frac_ff2(float2 Gh, float2 Gl, float2 rh,
                                         float2 rl, float dh, float dl,
                                         float2 &fh, float2 &fl,
                                         float2 &nf) {
  const float2 d2 = make_float2(dh, dh), l2 = make_float2(dl, dl);
  const float2 pn = fmul2(Gh, make_float2(-dh, -dh));  // -p, p = Gh dh
  const float2 pe = ffma2(Gh, d2, pn);                 // Gh dh - p
  const float2 t = fsub2(rh, pn);                      // two_sum(p, rh)
  const float2 bb = fadd2(t, pn);
  const float2 te = fsub2(fsub2(rh, bb), fadd2(pn, fsub2(t, bb)));
  float2 lo = fadd2(fadd2(pe, te), rl);
  lo = ffma2(Gh, l2, lo);
  lo = ffma2(Gl, d2, lo);
  nf = make_float2(rintf(t.x), rintf(t.y));
  const float2 t2 = fsub2(t, nf);  // exact
  fh = fadd2(t2, lo);
  fl = fsub2(lo, fsub2(fh, t2));
}

// sin(pi x) of two arguments at once: sinpi_reduced lane by lane
__device__ __forceinline__ float2 sinpi_reduced2(float2 x) {
  const float2 t = fmul2(x, x);
  float2 p = ffma2(make_float2(-6.941131045e-03f, -6.941131045e-03f), t,
                   make_float2(8.199509639e-02f, 8.199509639e-02f));
  p = ffma2(p, t, make_float2(-5.992401060e-01f, -5.992401060e-01f));
  p = ffma2(p, t, make_float2(2.550162271e+00f, 2.550162271e+00f));
  p = ffma2(p, t, make_float2(-5.167712735e+00f, -5.167712735e+00f));
  p = ffma2(p, t, make_float2(3.141592653e+00f, 3.141592653e+00f));
  return fmul2(x, p);
}

// sin(pi x) of two arguments at once for |x| <= ~0.55 with one FMA less:
// x * p(x^2), p the degree-4 least-squares fit of sin(pi x)/x in x^2 at 400
// Chebyshev nodes of [0, 0.56] (max relative error 2.7e-8 in exact
// arithmetic, a few ulp evaluated in FP32, as the degree-5 form)
__device__ __forceinline__ float2 sinpi_reduced2_d4(float2 x) {
  const float2 t = fmul2(x, x);
  float2 p = ffma2(make_float2(7.667203137e-02f, 7.667203137e-02f), t,
                   make_float2(-5.978266244e-01f, -5.978266244e-01f));
  p = ffma2(p, t, make_float2(2.550012410e+00f, 2.550012410e+00f));
  p = ffma2(p, t, make_float2(-5.167707502e+00f, -5.167707502e+00f));
  p = ffma2(p, t, make_float2(3.141592635e+00f, 3.141592635e+00f));
  return fmul2(x, p);
}

// y = N f - rint(N f) for two axes, f = fh + fl (double-float), N f formed
// exactly (two_prod) before the reduction; the negated products keep the
// roundings of the scalar form
__device__ __forceinline__ float2 sinc_arg2(float2 N2, float2 fh, float2 fl) {
  const float2 nN2 = make_float2(-N2.x, -N2.y);
  const float2 yh = fmul2(N2, fh);
  const float2 ye_neg = ffma2(nN2, fh, yh);       // -(N fh - yh)
  const float2 yl_neg = ffma2(nN2, fl, ye_neg);   // -(N fl + ye)
  const float2 rr = make_float2(rintf(yh.x), rintf(yh.y));
  return fsub2(fsub2(yh, rr), yl_neg);
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
      long long off =
          ((long long)(fl[0] - 1) * a.hn[1] + (fl[1] - 1)) * a.hn[2] +
          (fl[2] - 1);
      {
        const long long last = off + (3ll * a.hn[1] + 3) * a.hn[2] + 3;
        if (nb_idx(a.check, NB_SITE_STENCIL, last, table_size(a)) != last)
          off = 0;
      }
      float sum = 0.f;
      if (a.F4) {
        const float4 *b4 = a.F4 + off;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float si = 0.f;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float4 r = __ldg(b4 + ((long long)i * a.hn[1] + j) * a.hn[2]);
            float sj = wl[0] * r.x;
            sj = fmaf(wl[1], r.y, sj);
            sj = fmaf(wl[2], r.z, sj);
            sj = fmaf(wl[3], r.w, sj);
            si = fmaf(wk[j], sj, si);
          }
          sum = fmaf(wh[i], si, sum);
        }
        return sum;
      }
      const float *base = a.F + off;
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
    return __ldg(a.F + nb_idx(a.check, NB_SITE_F,
                              ((long long)n[0] * a.hn[1] + n[1]) * a.hn[2] +
                                  n[2],
                              table_size(a)));
  return a.defF;
}

}  // namespace nbgb
