// split_pixel.cuh -- the warp-per-pixel FP32-mixed Bragg-spot sum for
// Gaussian shapes, shared by the stand-alone kernel (spots_split.cu) and the
// serving kernel (serve.cu): table staging (split_stage), the FP64 set-up of
// one sub-pixel unit (split_unit) and the per-pixel sum of one warp
// (split_sum).  See spots_split.cu for the method.
#pragma once

#include "mixed_common.cuh"

namespace nbgb {

constexpr int kSplitWarps = 4;
constexpr int kSplitThreads = kSplitWarps * 32;
constexpr int kRing = 64;
constexpr int kMaxUnits = 32;
constexpr int kUnitFloats = 10;  // vh[3], vl[3], scal, df[3]
// per-lane item state, 9 float2: (G_hi, r_q) and (G_lo, r_lo) per axis,
// (n0_h, n0_k), (n0_l, scal), one unused.  Pairs halve the shared loads;
// the odd pair stride keeps distinct owners on distinct bank pairs unless
// they are 16 lanes apart.
constexpr int kStateStride = 18;
constexpr int kCandRing = 64;     // per-warp ring of (lane, source block)
constexpr int kSrcBlock = 8;      // sources per pruning block

struct SplitRing {
  float4 fw[kRing];  // f_h, f_k, f_l, weight: one 16-byte store / load
  int4 n[kRing];     // table-relative nearest index (h, k, l), unused
};
static_assert(sizeof(SplitRing) % 16 == 0, "rings stay 16-byte aligned");
static_assert(SRC32_DL % 2 == 0 && SRC32_W == SRC32_DL + 1 &&
                  SRC32_STRIDE % 2 == 0 && kUnitFloats % 2 == 0,
              "float2 reads of (delta_lo, w) and of the unit rows");

// ff_dot3 (mixed_common.cuh) with the double-float row stored as
// interleaved (hi, lo) pairs: the same operations, half the shared loads
__device__ __forceinline__ void ff_dot3_pairs(const float2 *A,
                                              const float *vh,
                                              const float *vl, float &gh,
                                              float &gl) {
  const float2 a0 = A[0], a1 = A[1], a2 = A[2];
  float p0, e0, p1, e1, p2, e2;
  two_prod(a0.x, vh[0], p0, e0);
  two_prod(a1.x, vh[1], p1, e1);
  two_prod(a2.x, vh[2], p2, e2);
  float s, t, s2, t2;
  two_sum(p0, p1, s, t);
  two_sum(s, p2, s2, t2);
  float lo = e0 + e1 + e2 + t + t2;
  lo = fmaf(a0.x, vl[0], lo);
  lo = fmaf(a1.x, vl[1], lo);
  lo = fmaf(a2.x, vl[2], lo);
  lo = fmaf(a0.y, vh[0], lo);
  lo = fmaf(a1.y, vh[1], lo);
  lo = fmaf(a2.y, vh[2], lo);
  fast_two_sum(s2, lo, gh, gl);
}

template <int INTERP>
__device__ __forceinline__ void eval_term(const SpotArgs &a,
                                          const SplitRing &q, int e,
                                          Kahan &acc) {
  const float4 fw = q.fw[e];
  const int4 ni = q.n[e];
  float fr[3] = {fw.x, fw.y, fw.z};
  int n[3] = {ni.x, ni.y, ni.z};
  float rad2 = a.N[0] * a.N[0] * fr[0] * fr[0];
  rad2 = fmaf(a.N[1] * a.N[1], fr[1] * fr[1], rad2);
  rad2 = fmaf(a.N[2] * a.N[2], fr[2] * fr[2], rad2);
  // fast exp: a few ulp for the significant terms (|argument| < ~20)
  float fl2 = a.N6 * __expf(-2.f * rad2 * (1.f / 0.63f));
  float fc;
  int fl[3];
  float x[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    int neg = fr[c] < 0.f;
    fl[c] = n[c] - neg;
    x[c] = neg ? 1.f + fr[c] : fr[c];
  }
  if (INTERP == 1 && a.C4 && fl[0] >= 1 && fl[0] + 2 < a.hn[0] &&
      fl[1] >= 1 && fl[1] + 2 < a.hn[1] && fl[2] >= 1 && fl[2] + 2 < a.hn[2]) {
    // the cell's tricubic polynomial, nested Horner in l, k, h (63 FMAs)
    const float4 *cp =
        a.C4 + (((long long)(fl[0] - 1) * (a.hn[1] - 3) + (fl[1] - 1)) *
                    (a.hn[2] - 3) + (fl[2] - 1)) * 16;
    float qa[4];
#pragma unroll
    for (int ia = 0; ia < 4; ++ia) {
      float pb[4];
#pragma unroll
      for (int ib = 0; ib < 4; ++ib) {
        float4 c4 = __ldg(cp + ia * 4 + ib);
        pb[ib] = fmaf(fmaf(fmaf(c4.w, x[2], c4.z), x[2], c4.y), x[2], c4.x);
      }
      qa[ia] = fmaf(fmaf(fmaf(pb[3], x[1], pb[2]), x[1], pb[1]), x[1], pb[0]);
    }
    fc = fmaf(fmaf(fmaf(qa[3], x[0], qa[2]), x[0], qa[1]), x[0], qa[0]);
  } else {
    fc = fcell_f32<INTERP>(a, n, fr);
  }
  acc.add(fc * fc * fl2 * fw.w);
}

// Per-block view of one shot's staged tables in shared memory and the
// constants derived from them.
struct SplitBlock {
  const float2 *ax2;  // [PM][9] (hi, lo) pairs
  const float *src, *blk, *dh;
  float *unit_base, *state_base;
  int *cring_base;
  SplitRing *rings;
  int PM, S, nblk, sstep;
  float u0h, u0l, cwide, dmin, dmax, dmarg, inv_step;
  float cmarg[3];
  bool iv_ok, even;
};

// Stages a shot's tables (double-float axes [PM][9], interleaved into
// (hi, lo) pairs, and source rows [S][12]) into the dynamic shared memory
// `sms` and derives the pruning constants.  Called by every thread of the
// block.
__device__ __forceinline__ void split_stage(SplitBlock &b, float *sms,
                                            const SpotArgs &a,
                                            const float *axh, const float *axl,
                                            const float *src32, int PM, int S,
                                            float u0h, float u0l) {
  float2 *s_ax2 = reinterpret_cast<float2 *>(sms);
  float *s_src = sms + 2 * PM * 9;
  float *s_unit = s_src + S * SRC32_STRIDE;  // [warp][unit][kUnitFloats]
  // the rings hold float4s: 16-byte aligned base
  size_t ring_off =
      ((size_t)(s_unit + kSplitWarps * kMaxUnits * kUnitFloats - sms) *
           sizeof(float) + 15) & ~(size_t)15;
  SplitRing *rings = reinterpret_cast<SplitRing *>(
      reinterpret_cast<char *>(sms) + ring_off);
  float *s_state = reinterpret_cast<float *>(rings + kSplitWarps);
  int *s_cring =
      reinterpret_cast<int *>(s_state + kSplitWarps * 32 * kStateStride);
  float *s_blk = reinterpret_cast<float *>(s_cring + kSplitWarps * kCandRing);
  const int nblk = (S + kSrcBlock - 1) / kSrcBlock;
  float *s_dh = s_blk + 2 * nblk;  // delta_hi of every source, contiguous
  for (int i = threadIdx.x; i < PM * 9; i += blockDim.x)
    s_ax2[i] = make_float2(axh[i], axl[i]);
  for (int i = threadIdx.x; i < S * SRC32_STRIDE; i += blockDim.x)
    s_src[i] = src32[i];
  __syncthreads();
  // delta_hi range of every block of kSrcBlock sources (the pruning test)
  for (int bb = threadIdx.x; bb < nblk; bb += blockDim.x) {
    float mn = 3.0e38f, mx = -3.0e38f;
    for (int k = bb * kSrcBlock; k < S && k < (bb + 1) * kSrcBlock; ++k) {
      float d = s_src[k * SRC32_STRIDE + SRC32_DH];
      mn = fminf(mn, d);
      mx = fmaxf(mx, d);
    }
    s_blk[2 * bb] = mn;
    s_blk[2 * bb + 1] = mx;
  }
  for (int k = threadIdx.x; k < S; k += blockDim.x)
    s_dh[k] = s_src[k * SRC32_STRIDE + SRC32_DH];
  __syncthreads();
  // exact intervals need delta_hi in ascending order (the library sorts the
  // sources; a caller of the allocation-free entry may not)
  int unsorted = 0;
  for (int k = threadIdx.x; k + 1 < S; k += blockDim.x)
    unsorted |= s_dh[k] > s_dh[k + 1];
  const bool dh_sorted = __syncthreads_or(unsorted) == 0;
  b.ax2 = s_ax2;
  b.src = s_src;
  b.blk = s_blk;
  b.dh = s_dh;
  b.unit_base = s_unit;
  b.state_base = s_state;
  b.cring_base = s_cring;
  b.rings = rings;
  b.PM = PM;
  b.S = S;
  b.nblk = nblk;
  b.u0h = u0h;
  b.u0l = u0l;
  // a widened cut for the conservative tests: every surviving term has
  // sum N^2 f^2 <= cutg < cwide, so |f_x| <= sqrt(cwide) / N_x
  const float cutg = kGaussCut * 0.63f;
  b.cwide = cutg * 1.02f + 1e-4f;
  for (int x = 0; x < 3; ++x) b.cmarg[x] = sqrtf(b.cwide) / a.N[x];
  // exact delta-intervals per lattice point need the ellipsoids of
  // neighbouring lattice points to be disjoint: sqrt(cwide)/N < 1/2
  b.iv_ok = dh_sorted && b.cmarg[0] < 0.49f && b.cmarg[1] < 0.49f &&
            b.cmarg[2] < 0.49f;
  b.dmin = S > 0 ? s_dh[0] : 0.f;
  b.dmax = S > 0 ? s_dh[S - 1] : 0.f;
  b.dmarg = 1e-3f * (b.dmax - b.dmin) / (float)(S > 1 ? S - 1 : 1);
  int sstep = 1;
  while (sstep * 2 <= S) sstep *= 2;
  b.sstep = sstep;
  // nearly even delta spacing (an equispaced spectrum): the position of a
  // bound in the table is then guessed from the spacing and corrected by a
  // step or two, instead of a binary search
  const float step = S > 1 ? (b.dmax - b.dmin) / (float)(S - 1) : 0.f;
  int uneven = !(step > 0.f);
  for (int k = threadIdx.x; k < S && !uneven; k += blockDim.x)
    uneven |= !(fabsf(s_dh[k] - fmaf((float)k, step, b.dmin)) <= step);
  b.even = __syncthreads_or(uneven) == 0;
  b.inv_step = b.even ? 1.f / step : 0.f;
}

// k1 = #{k : delta_k < lo} and k2 = #{k : delta_k <= hi} in the ascending
// table dh[0..S): from a guess, walk down while the entry below is on the
// wrong side, then up while the entry above is.  Exact for any guess in
// [0, S]; the guess only sets the number of steps.
__device__ __forceinline__ int count_below(const float *dh, int S, int k,
                                           float lo) {
  while (k > 0 && dh[k - 1] >= lo) --k;
  while (k < S && dh[k] < lo) ++k;
  return k;
}
__device__ __forceinline__ int count_at_most(const float *dh, int S, int k,
                                             float hi) {
  while (k > 0 && dh[k - 1] > hi) --k;
  while (k < S && dh[k] <= hi) ++k;
  return k;
}
__device__ __forceinline__ int guess_index(float x, float dmin, float inv,
                                           int S) {
  // fmaxf/fminf also map a NaN to 0
  return (int)fminf(fmaxf(ceilf((x - dmin) * inv), 0.f), (float)S);
}

// Geometry of sub-pixel unit u (subpixel i, j, sensor layer t) of pixel
// (s, f) of panel P into ud[kUnitFloats]: v = d - i0 as double-float,
// omega cap (times the polarization for one beam direction), and d in FP32.
template <int HASDIV>
__device__ __forceinline__ void split_unit(const SpotArgs &a,
                                           const DevPanel &P, int s, int f,
                                           int u, float *ud) {
  const int os = a.os;
  const float kahn = a.kahn;
  int t = u % a.T, ij = u / a.T, i = ij / os, j = ij % os;
  float vh[3], vl[3], df[3], omega;
  // FP64 here (one rsqrt, products): in these kernels the FP32 pipe is the
  // busy one and the FP64 work of a batch of units overlaps with it; the
  // double-float form (unit_geometry_ff, which the thread-per-pixel kernel
  // uses) measured slower here
  {
    const double px = P.px, inv_os = 1.0 / os;
    double cf = (f + (i + 0.5) * inv_os) * px,
           cs = (s + (j + 0.5) * inv_os) * px, cn = t * a.dt;
    double pos[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      pos[c] = P.origin[c] + cf * P.fdir[c] + cs * P.sdir[c] +
               cn * P.ndir[c];
    const double inv = rsqrt(dot3d_m(pos, pos));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double d = pos[c] * inv, v = d - a.i0[c];
      vh[c] = (float)v;
      vl[c] = (float)(v - (double)vh[c]);
      df[c] = (float)d;
    }
    omega = (float)(px * px * dot3d_m(P.ndir, pos) * (inv * inv * inv));
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ud[c] = vh[c];
    ud[3 + c] = vl[c];
    ud[7 + c] = df[c];
  }
  float cap = 1.f;
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
  ud[6] = scal;
}

// The sum, without the prefactor, of the pixel whose U sub-pixel units are
// already in `unit` (split_unit), computed by the calling warp (all 32
// lanes); every lane returns the same value.  Adds the number of evaluated
// terms to `evals`.
template <int INTERP, int HASDIV>
__device__ __forceinline__ double split_sum(const SpotArgs &a,
                                            const SplitBlock &b,
                                            const float *unit,
                                            unsigned long long &evals) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int PM = b.PM, S = b.S, nblk = b.nblk, sstep = b.sstep;
  const float2 *s_ax2 = b.ax2;
  const float *s_src = b.src, *s_blk = b.blk,
              *s_dh = b.dh;
  SplitRing &q = b.rings[warp];
  float *st = b.state_base + warp * 32 * kStateStride;
  int *cring = b.cring_base + warp * kCandRing;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int U = a.os * a.os * a.T, items = U * PM;
  const float cutg = kGaussCut * 0.63f;
  const float kahn = a.kahn;
  const float N2[3] = {a.N[0] * a.N[0], a.N[1] * a.N[1], a.N[2] * a.N[2]};
  const float cwide = b.cwide;
  const float cmarg[3] = {b.cmarg[0], b.cmarg[1], b.cmarg[2]};
  const bool iv_ok = b.iv_ok;
  const float dmin = b.dmin, dmax = b.dmax, dmarg = b.dmarg;
  const bool even = b.even;
  const float inv_step = b.inv_step;
  const float u0h = b.u0h, u0l = b.u0l;

  // ---- 2./3. scan the steps, evaluate surviving terms 32 at a time
  Kahan acc;
  int head = 0, tail = 0;
  for (int base = 0; base < items; base += 32) {
    int it = base + lane;
    bool valid = it < items;
    int u = valid ? it / PM : 0, pm = valid ? it - u * PM : 0;
    const float *ud = unit + u * kUnitFloats;
    // vh[3], vl[3], scal as four float2 loads (unit rows are 8-byte aligned)
    const float2 *u2 = reinterpret_cast<const float2 *>(ud);
    const float2 p0 = u2[0], p1 = u2[1], p2 = u2[2], p3 = u2[3];
    float vh[3] = {p0.x, p0.y, p1.x}, vl[3] = {p1.y, p2.x, p2.y};
    float scal = p3.x;
    float Gh[3], Gl[3], rq[3], rl[3], n0[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      ff_dot3_pairs(s_ax2 + pm * 9 + 3 * x, vh, vl, Gh[x], Gl[x]);
      float qh, qe;
      two_prod(Gh[x], u0h, qh, qe);
      float ql = fmaf(Gh[x], u0l, fmaf(Gl[x], u0h, qe));
      n0[x] = rintf(qh);
      float rh, rl0;
      two_sum(__fsub_rn(qh, n0[x]), ql, rh, rl0);
      // r_hi on a 2^-21 grid: r_hi - n is then exact for |n| < 7
      rq[x] = __fmul_rn(rintf(__fmul_rn(rh, 2097152.f)), 1.f / 2097152.f);
      rl[x] = rl0 + __fsub_rn(rh, rq[x]);
    }
    if (HASDIV) {
      for (int k = 0; k < S; ++k) {
        const float *src = s_src + k * SRC32_STRIDE;
        const float dh = src[SRC32_DH];
        // cut test on the cheap offset t - rint(t) (error ~1 ulp of t, which
        // only moves terms ~1e-38 below the peak across the cut)
        float tq[3], nf[3], fr[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          tq[x] = fmaf(Gh[x], dh, rq[x]);
          if (HASDIV && valid) tq[x] -= __ldg(a.divh + ((size_t)pm * S + k) * 3 + x);
          nf[x] = rintf(tq[x]);
          fr[x] = tq[x] - nf[x];
        }
        float rad2 = N2[0] * fr[0] * fr[0];
        rad2 = fmaf(N2[1] * fr[1], fr[1], rad2);
        rad2 = fmaf(N2[2] * fr[2], fr[2], rad2);
        bool hit = valid && rad2 <= cutg;
        unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m == 0u) continue;
        if (hit) {
          // the precise offset: G_hi d_hi + (r_q - n) in one rounding (r_q
          // on a 2^-21 grid makes r_q - n exact) plus the small terms
          const float dl = src[SRC32_DL];
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            float sx = fmaf(Gh[x], dh, __fsub_rn(rq[x], nf[x]));
            float c = fmaf(Gh[x], dl, fmaf(Gl[x], dh, rl[x]));
            fr[x] = sx + c;
            if (HASDIV) {
              // the divergence term moves h after the rint: re-centre
              size_t e = ((size_t)pm * S + k) * 3 + x;
              fr[x] -= __ldg(a.divh + e) + __ldg(a.divl + e);
              float n2 = rintf(fr[x]);
              fr[x] -= n2;
              nf[x] += n2;
            }
          }
          int e = (tail + __popc(m & lt_mask)) & (kRing - 1);
          float w = src[SRC32_W] * scal;
          if (HASDIV) {
            const float *df = ud + 7, *dir = src + SRC32_DIR,
                        *ev = src + SRC32_E, *bv = src + SRC32_B;
            float c2 = df[0] * dir[0] + df[1] * dir[1] + df[2] * dir[2];
            float x = df[0] * ev[0] + df[1] * ev[1] + df[2] * ev[2];
            float y = df[0] * bv[0] + df[1] * bv[1] + df[2] * bv[2];
            w *= 0.5f * (1.f + c2 * c2 - kahn * (x * x - y * y));
          }
          q.fw[e] = make_float4(fr[0], fr[1], fr[2], w);
          q.n[e] = make_int4(__float2int_rn(n0[0] + nf[0]) - a.hmin[0],
                             __float2int_rn(n0[1] + nf[1]) - a.hmin[1],
                             __float2int_rn(n0[2] + nf[2]) - a.hmin[2], 0);
        }
        tail += __popc(m);
        if (tail - head >= 32) {
          __syncwarp();
          eval_term<INTERP>(a, q, (head + lane) & (kRing - 1), acc);
          head += 32;
          __syncwarp();
        }
      }
    } else {
      // ---- pruned scan: h_x = G_x delta + r_x is linear in delta, so a
      // block of sources whose delta range [dmin, dmax] keeps some axis
      // farther than sqrt(cut)/N_x from every integer holds no surviving
      // term.  Surviving (lane, block) pairs go into a ring; the warp
      // then runs 4 blocks x 8 sources = 32 steps at a time.
      float2 *my = reinterpret_cast<float2 *>(st + lane * kStateStride);
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        my[x] = make_float2(Gh[x], rq[x]);
        my[3 + x] = make_float2(Gl[x], rl[x]);
      }
      my[6] = make_float2(n0[0], n0[1]);
      my[7] = make_float2(n0[2], scal);
      __syncwarp();
      int ch = 0, ct = 0;
      auto run_cands = [&](int nc) {
        // ring entry: owner lane | first source << 5 | count << 16
        const int ci = lane >> 3, kk = lane & 7;
        bool ok = ci < nc;
        int ent = ok ? cring[(ch + ci) & (kCandRing - 1)] : 0;
        int own = ent & 31, k0 = (ent >> 5) & 2047, cnt = (ent >> 16) & 15;
        int k = k0 + kk;
        ok = ok && kk < cnt && k < S;
        const float2 *o =
            reinterpret_cast<const float2 *>(st + own * kStateStride);
        const float dh = s_dh[ok ? k : 0];
        float fr[3], nf[3];
        float2 gr[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          gr[x] = o[x];  // (G_hi, r_q)
          float tq = fmaf(gr[x].x, dh, gr[x].y);
          nf[x] = rintf(tq);
          fr[x] = tq - nf[x];
        }
        float rad2 = N2[0] * fr[0] * fr[0];
        rad2 = fmaf(N2[1] * fr[1], fr[1], rad2);
        rad2 = fmaf(N2[2] * fr[2], fr[2], rad2);
        bool hit = ok && rad2 <= cutg;
        unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m == 0u) return;
        if (hit) {
          // (delta_lo, w) of source k in one load
          const float2 dlw = *reinterpret_cast<const float2 *>(
              s_src + k * SRC32_STRIDE + SRC32_DL);
          const float dl = dlw.x;
          int e = (tail + __popc(m & lt_mask)) & (kRing - 1);
          const float2 n01 = o[6], n2s = o[7];
          const float n0o[3] = {n01.x, n01.y, n2s.x};
          float f[3];
          int nn[3];
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            const float2 gl = o[3 + x];  // (G_lo, r_lo)
            float sx = fmaf(gr[x].x, dh, __fsub_rn(gr[x].y, nf[x]));
            float c = fmaf(gr[x].x, dl, fmaf(gl.x, dh, gl.y));
            f[x] = sx + c;
            nn[x] = __float2int_rn(n0o[x] + nf[x]) - a.hmin[x];
          }
          q.fw[e] = make_float4(f[0], f[1], f[2], dlw.y * n2s.y);
          q.n[e] = make_int4(nn[0], nn[1], nn[2], 0);
        }
        tail += __popc(m);
        if (tail - head >= 32) {
          __syncwarp();
          eval_term<INTERP>(a, q, (head + lane) & (kRing - 1), acc);
          head += 32;
          __syncwarp();
        }
      };
      // lattice points the item's sweep can come near: per axis the
      // integers within sqrt(cwide)/N_x of [h(dmin), h(dmax)]
      int ml[3] = {0, 0, 0}, nm[3] = {0, 0, 0}, ncomb = 0;
      if (iv_ok && valid) {
        ncomb = 1;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          float u = fmaf(Gh[x], dmin, rq[x]), v = fmaf(Gh[x], dmax, rq[x]);
          ml[x] = (int)ceilf(fminf(u, v) - cmarg[x]);
          nm[x] = (int)floorf(fmaxf(u, v) + cmarg[x]) - ml[x] + 1;
          if (nm[x] < 0) nm[x] = 0;
          ncomb *= nm[x];
        }
      }
      if (iv_ok && __all_sync(0xffffffffu, ncomb <= 8)) {
        // exact intervals: for lattice point m the exponent sum along
        // the sweep is A d^2 + 2 B d + C, below cwide on one interval
        const int maxc = (int)__reduce_max_sync(0xffffffffu, (unsigned)ncomb);
        for (int c = 0; c < maxc; ++c) {
          int k1 = 0, k2 = 0;
          if (c < ncomb) {
            float dx[3];
            int cc = c;
#pragma unroll
            for (int x = 0; x < 3; ++x) {
              int mx = ml[x] + cc % nm[x];
              cc /= nm[x];
              dx[x] = rq[x] - (float)mx;  // exact: r_q on a 2^-21 grid
            }
            float A = N2[0] * Gh[0] * Gh[0];
            A = fmaf(N2[1] * Gh[1], Gh[1], A);
            A = fmaf(N2[2] * Gh[2], Gh[2], A);
            float B = N2[0] * Gh[0] * dx[0];
            B = fmaf(N2[1] * Gh[1], dx[1], B);
            B = fmaf(N2[2] * Gh[2], dx[2], B);
            float C0 = N2[0] * dx[0] * dx[0];
            C0 = fmaf(N2[1] * dx[1], dx[1], C0);
            C0 = fmaf(N2[2] * dx[2], dx[2], C0);
            if (A > 0.f) {
              float disc = fmaf(B, B, -A * (C0 - cwide));
              if (disc >= 0.f) {
                float sq = sqrtf(disc);
                float lo = (-B - sq) / A, hi = (-B + sq) / A;
                float mg = 1e-4f * (fabsf(lo) + fabsf(hi)) + dmarg;
                lo -= mg;
                hi += mg;
                // k1 = #{delta < lo}, k2 = #{delta <= hi} (sorted table)
                if (even) {
                  k1 = count_below(s_dh, S, guess_index(lo, dmin, inv_step, S),
                                   lo);
                  k2 = count_at_most(s_dh, S,
                                     guess_index(hi, dmin, inv_step, S), hi);
                } else {
                  for (int st = sstep; st > 0; st >>= 1) {
                    if (k1 + st <= S && s_dh[k1 + st - 1] < lo) k1 += st;
                    if (k2 + st <= S && s_dh[k2 + st - 1] <= hi) k2 += st;
                  }
                }
              }
            } else if (C0 <= cwide) {
              k2 = S;  // the sweep does not move: all or nothing
            }
          }
          const int nch = k2 > k1 ? (k2 - k1 + kSrcBlock - 1) / kSrcBlock : 0;
          const int maxch =
              (int)__reduce_max_sync(0xffffffffu, (unsigned)nch);
          for (int j = 0; j < maxch; ++j) {
            bool has = j < nch;
            unsigned mm = __ballot_sync(0xffffffffu, has);
            if (has) {
              int st0 = k1 + j * kSrcBlock;
              int cnt = min(kSrcBlock, k2 - st0);
              cring[(ct + __popc(mm & lt_mask)) & (kCandRing - 1)] =
                  lane | (st0 << 5) | (cnt << 16);
            }
            ct += __popc(mm);
            __syncwarp();
            while (ct - ch >= 4) {
              run_cands(4);
              ch += 4;
            }
          }
        }
      } else {
        for (int b = 0; b < nblk; ++b) {
          bool pass = false;
          if (valid) {
            const float dmn = s_blk[2 * b], dmx = s_blk[2 * b + 1];
            pass = true;
#pragma unroll
            for (int x = 0; x < 3; ++x) {
              float u = fmaf(Gh[x], dmn, rq[x]), v = fmaf(Gh[x], dmx, rq[x]);
              float lo = fminf(u, v) - cmarg[x],
                    hi = fmaxf(u, v) + cmarg[x];
              pass = pass && floorf(hi) >= ceilf(lo);
            }
          }
          unsigned m = __ballot_sync(0xffffffffu, pass);
          if (m == 0u) continue;
          if (pass) {
            int st0 = b * kSrcBlock;
            int cnt = min(kSrcBlock, S - st0);
            cring[(ct + __popc(m & lt_mask)) & (kCandRing - 1)] =
                lane | (st0 << 5) | (cnt << 16);
          }
          ct += __popc(m);
          __syncwarp();
          while (ct - ch >= 4) {
            run_cands(4);
            ch += 4;
          }
        }
      }
      if (ct > ch) {
        run_cands(ct - ch);
        ch = ct;
      }
      __syncwarp();  // the state area is rewritten by the next round
    }
  }
  __syncwarp();
  if (lane < tail - head)
    eval_term<INTERP>(a, q, (head + lane) & (kRing - 1), acc);
  evals += tail;
  __syncwarp();

  // ---- 4. warp reduction in float-float: each lane's compensated sum is
  // the pair (s, -c); pairs are added with error-free transformations (so
  // the butterfly gives every lane the same pair) and turned into FP64
  // once.  FP64 instructions run at 1/64 of the FP32 rate on this part and
  // issue per warp, so a per-pixel FP64 tree would cost as much as a
  // pixel's sum when the pixel has few steps.
  float hi, lo;
  fast_two_sum(acc.s, -acc.c, hi, lo);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    float sh, se;
    two_sum(hi, h2, sh, se);
    se += lo + l2;
    fast_two_sum(sh, se, hi, lo);
  }
  __syncwarp();
  return (double)hi + (double)lo;
}

}  // namespace nbgb
