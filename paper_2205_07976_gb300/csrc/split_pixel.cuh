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
constexpr int kMaxUnits = 32;
constexpr int kUnitFloats = 10;  // vh[3], vl[3], scal, df[3]
constexpr int kSrcBlock = 8;     // sources per pruning block
// Per-warp ring of source intervals.  An entry is one (item, source range)
// pair that can hold surviving terms, with a copy of its item's state, so
// that entries outlive the item batch that pushed them.  Pending entries
// never exceed 31 (each holds an unconsumed source) plus the 32 a push adds.
constexpr int kEntries = 64;

// Two kinds of entry.  An interval entry belongs to one lattice point m of
// the item's sweep: every surviving step of it has m as its nearest
// integer, so the entry holds r_q - (m - n0) in place of r_q and m's table
// index, and a step's offset needs no rounding.  A block entry (pruning by
// source blocks, or sources of different directions) holds r_q and n0, and
// each step rounds to its nearest integer.
struct SplitEntry {
  float4 a;  // G_hi h, G_hi k, r h, r k      (r = r_q, or r_q - (m - n0))
  float4 b;  // G_lo h, G_lo k, r_lo h, r_lo k
  float4 c;  // G_hi l, r l, G_lo l, r_lo l
  float4 d;  // n0 h, n0 k, n0 l (floats), or for m (int bits) its table
             // index, or with tricubic cell polynomials ci0, the index
             // packed (10 bits per axis, plus 1) and pk (entry_cell_data);
             // and omega cap pol of the unit
  int4 m;    // first source, count, position of the first source in the
             // pixel's sequence of (entry, source) pairs,
             // pm | unit << 16 | interval entry << 31
};
constexpr int kIntervalEntry = 1 << 31;
static_assert(sizeof(SplitEntry) % 16 == 0, "entries stay 16-byte aligned");
static_assert(SRC32_DL == 0 && SRC32_W == 1 && SRC32_DH == 2 &&
                  SRC32_STRIDE % 4 == 0 && kUnitFloats % 2 == 0,
              "one float4 read of (delta_lo, w, delta_hi, .) per source "
              "and float2 reads of the unit rows");

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

// Per-warp cache of cell polynomials in shared memory.  The terms of one
// evaluation pass almost always lie around a single lattice point n, in the
// cells n - {0,1}^3, and those 8 cells have distinct parities (the low bit
// of each corner index).  So the cache has one slot per parity, and chunk k
// (float4) of slot p sits at float4 k * kCellSlots + p: the same chunk of
// every slot lies in one 128-byte row of shared-memory banks, and one
// 16-byte load of chunk k by all lanes is a single shared-memory wavefront
// whatever mix of slots the lanes read (lanes on one slot get a
// broadcast).  A global 16-byte load delivers 128 bytes per wavefront
// whether the lanes' addresses coincide or not, so reading the 256
// coefficient bytes of each term from global memory costs 2 wavefronts per
// term; from the cache it costs 1/2.
constexpr int kCellSlots = 8;
constexpr int kCellChunks = 16;  // float4 per cell polynomial

// A cell's tricubic polynomial at x (cell coordinates in [0, 1)): nested
// Horner in l, k, h, the z and y chains of the powers x^(2P) and x^(2P+1)
// side by side in packed FMAs (30 packed + 3 scalar FMAs for the 63 of
// the scalar form, with the same roundings); chunk q of the coefficients
// (the layout of SpotArgs::C4) at cp[q * stride], read from shared memory
// (SHARED) or through the read-only path.
template <bool SHARED>
__device__ __forceinline__ float cell_horner(const float4 *cp, int stride,
                                             const float x[3]) {
  const float2 z2 = make_float2(x[2], x[2]), y2 = make_float2(x[1], x[1]);
  float2 q[2];
#pragma unroll
  for (int P = 0; P < 2; ++P) {
    float2 pb[4];
#pragma unroll
    for (int ib = 0; ib < 4; ++ib) {
      const int q0 = (P * 4 + ib) * 2;
      const float4 A = SHARED ? cp[q0 * stride] : __ldg(cp + q0 * stride);
      const float4 B =
          SHARED ? cp[(q0 + 1) * stride] : __ldg(cp + (q0 + 1) * stride);
      float2 v = ffma2(make_float2(A.x, A.y), z2, make_float2(A.z, A.w));
      v = ffma2(v, z2, make_float2(B.x, B.y));
      pb[ib] = ffma2(v, z2, make_float2(B.z, B.w));
    }
    q[P] = ffma2(ffma2(ffma2(pb[3], y2, pb[2]), y2, pb[1]), y2, pb[0]);
  }
  // q[P] = (C(x^(2P)) part, C(x^(2P+1)) part); Horner in x
  return fmaf(fmaf(fmaf(q[1].y, x[0], q[1].x), x[0], q[0].y), x[0], q[0].x);
}

// n[2] of a term whose index is still packed (interval entries with cell
// polynomials): n[0] then holds the packed index of SplitEntry::d.y
constexpr int kPackedIndex = -0x40000000;

// The cell of a tricubic term: whether its 4x4x4 stencil lies inside the
// table (tri), the cell's index in the polynomial table (ci), its parity
// slot in the cache (par) and the coordinates x in [0, 1) within the cell.
struct CellRef {
  bool tri;
  int ci, par;
  float x[3];
};

// The cell of a step with fractional offset fr and table-relative nearest
// index n: its stencil starts at fl - 1, fl = n - (fr < 0) per axis.
template <int INTERP>
__device__ __forceinline__ void cell_of(const SpotArgs &a, bool hit,
                                        const float fr[3], const int n[3],
                                        CellRef &c) {
  int fl[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int neg = fr[k] < 0.f;
    fl[k] = n[k] - neg;
    c.x[k] = neg ? 1.f + fr[k] : fr[k];
  }
  // the 4x4x4 stencil fl - 1 .. fl + 2 inside the table
  c.tri = INTERP == 1 && hit && a.C4 &&
          (unsigned)(fl[0] - 1) < (unsigned)(a.hn[0] - 3) &&
          (unsigned)(fl[1] - 1) < (unsigned)(a.hn[1] - 3) &&
          (unsigned)(fl[2] - 1) < (unsigned)(a.hn[2] - 3);
  c.ci = 0;
  c.par = 0;
  if (c.tri) {
    c.ci = ((fl[0] - 1) * (a.hn[1] - 3) + (fl[1] - 1)) * (a.hn[2] - 3) +
           (fl[2] - 1);
    c.par = (fl[0] & 1) | ((fl[1] & 1) << 1) | ((fl[2] & 1) << 2);
  }
}

// Cell data of an interval entry's lattice point m (table-relative index
// nt), computed once per entry: ci0 = the index of the cell whose stencil
// starts at nt - 1; pk = the parity of nt (bits 0-2) and, in bits 3-10,
// for each sign pattern s of a step's offset (bit k: f_k < 0, which moves
// the stencil one node down along axis k) whether that stencil lies inside
// the table.  A step's cell is then ci0 minus the strides its pattern
// selects, with parity pk ^ s.
__device__ __forceinline__ void entry_cell_data(const SpotArgs &a,
                                                const int nt[3], int &ci0,
                                                int &pk) {
  const int H1 = a.hn[1] - 3, H2 = a.hn[2] - 3;
  ci0 = ((nt[0] - 1) * H1 + (nt[1] - 1)) * H2 + (nt[2] - 1);
  // sign pattern s has bit k set when axis k moves down
  const unsigned pos_bits[3] = {0x55u, 0x33u, 0x0Fu};
  unsigned ok = 0xFFu;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const unsigned span = (unsigned)(a.hn[k] - 3);
    const bool up = (unsigned)(nt[k] - 1) < span;    // f_k >= 0
    const bool down = (unsigned)(nt[k] - 2) < span;  // f_k < 0
    ok &= (up ? pos_bits[k] : 0u) | (down ? (~pos_bits[k] & 0xFFu) : 0u);
  }
  pk = (nt[0] & 1) | ((nt[1] & 1) << 1) | ((nt[2] & 1) << 2) | (int)(ok << 3);
}

__device__ __forceinline__ void cell_of_entry(const SpotArgs &a, bool hit,
                                              const float fr[3], int ci0,
                                              int pk, CellRef &c) {
  const int s = (fr[0] < 0.f) | ((fr[1] < 0.f) << 1) | ((fr[2] < 0.f) << 2);
#pragma unroll
  for (int k = 0; k < 3; ++k) c.x[k] = fr[k] < 0.f ? 1.f + fr[k] : fr[k];
  const int H2 = a.hn[2] - 3;
  c.tri = hit && ((pk >> (3 + s)) & 1);
  c.ci = ci0 - ((s & 1) ? (a.hn[1] - 3) * H2 : 0) - ((s & 2) ? H2 : 0) -
         ((s >> 2) & 1);
  c.par = (pk & 7) ^ s;
}

// The term F_cell^2 F_latt^2 w of a lane whose step survived the cut (`hit`),
// given its fractional offset fr, table-relative nearest index n, cell c
// and exponent sum rad2 = sum N^2 fr^2.  Called
// by all 32 lanes of the warp: missing cells are loaded into the cache by
// the whole warp (one coalesced 256-byte read per cell).  A lane whose
// parity slot ends up holding another cell (two lattice points in one pass)
// reads its cell from global memory instead.
template <int INTERP>
__device__ __forceinline__ float term_value(const SpotArgs &a, bool hit,
                                            const CellRef &c,
                                            const float fr[3], const int n[3],
                                            float rad2, float w,
                                            float4 *cache, int *tags) {
  // fast exp: a few ulp for the significant terms (|argument| < ~20)
  const float fl2 = a.N6 * __expf(-2.f * rad2 * (1.f / 0.63f));
  bool cached = false;
  if (INTERP == 1) {
    const int lane = threadIdx.x & 31;
    unsigned miss = __ballot_sync(0xffffffffu, c.tri && tags[c.par] != c.ci);
    if (miss == 0u) {
      cached = c.tri;
    } else {
      unsigned handled = 0u;
      while (miss) {
        // load the cell of the first missing lane into its parity slot; each
        // slot is loaded at most once per pass
        const int src = __ffs(miss) - 1;
        const int sp = __shfl_sync(0xffffffffu, c.par, src);
        const int sci = __shfl_sync(0xffffffffu, c.ci, src);
        const float2 v = __ldg(
            reinterpret_cast<const float2 *>(
                a.C4 + (size_t)nb_idx(a.check, NB_SITE_CELL, sci,
                                      cell_count(a)) *
                           kCellChunks) +
            lane);
        reinterpret_cast<float2 *>(
            cache)[((lane >> 1) * kCellSlots + sp) * 2 + (lane & 1)] = v;
        __syncwarp();
        if (lane == 0) tags[sp] = sci;
        __syncwarp();
        handled |= 1u << sp;
        miss = __ballot_sync(0xffffffffu, c.tri && !((handled >> c.par) & 1u) &&
                                              tags[c.par] != c.ci);
      }
      cached = c.tri && tags[c.par] == c.ci;
    }
  }
  float fc = 0.f;
  if (cached) {
    fc = cell_horner<true>(cache + c.par, kCellSlots, c.x);
  } else if (c.tri) {
    fc = cell_horner<false>(
        a.C4 + (size_t)nb_idx(a.check, NB_SITE_CELL, c.ci, cell_count(a)) *
                   kCellChunks,
        1, c.x);
  } else if (hit) {
    int nn[3] = {n[0], n[1], n[2]};
    if (n[2] == kPackedIndex) {
      nn[0] = (n[0] & 1023) - 1;
      nn[1] = ((n[0] >> 10) & 1023) - 1;
      nn[2] = ((n[0] >> 20) & 1023) - 1;
    }
    fc = fcell_f32<INTERP>(a, nn, fr);
  }
  return fc * fc * fl2 * w;
}

// Per-block view of one shot's staged tables in shared memory and the
// constants derived from them.
struct SplitBlock {
  const float2 *ax2;  // [PM][9] (hi, lo) pairs
  const float *src, *blk, *dh;
  float *unit_base;
  SplitEntry *ent_base;  // [warp][kEntries]
  float4 *cell_cache;    // [warp][kCellChunks][kCellSlots]
  int *cell_tags;        // [warp][kCellSlots], -1 = empty
  int PM, S, nblk, sstep;
  float u0h, u0l, cwide, dmin, dmax, dmarg, inv_step;
  float cmarg[3];
  bool iv_ok, even;
};

// Bytes of dynamic shared memory split_stage lays out for PM orientations
// and S sources.
__host__ __device__ inline int split_axes_floats(int PM) {
  return (2 * PM * 9 + 3) & ~3;  // the source rows after it 16-byte aligned
}

__host__ __device__ inline size_t split_smem_layout(int PM, int S) {
  const int nblk = (S + kSrcBlock - 1) / kSrcBlock;
  size_t off = (size_t)(split_axes_floats(PM) + S * SRC32_STRIDE +
                        kSplitWarps * kMaxUnits * kUnitFloats) *
               sizeof(float);
  off = (off + 15) & ~(size_t)15;
  off += (size_t)kSplitWarps * kEntries * sizeof(SplitEntry);
  off += (size_t)kSplitWarps * kCellChunks * kCellSlots * sizeof(float4);
  off += (size_t)(2 * nblk + S) * sizeof(float);
  off += (size_t)kSplitWarps * kCellSlots * sizeof(int);
  return off;
}

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
  float *s_src = sms + split_axes_floats(PM);
  float *s_unit = s_src + S * SRC32_STRIDE;  // [warp][unit][kUnitFloats]
  // entries and cache hold float4s: 16-byte aligned base
  const size_t ent_off =
      ((size_t)(s_unit + kSplitWarps * kMaxUnits * kUnitFloats - sms) *
           sizeof(float) + 15) & ~(size_t)15;
  SplitEntry *s_ent = reinterpret_cast<SplitEntry *>(
      reinterpret_cast<char *>(sms) + ent_off);
  float4 *s_cache = reinterpret_cast<float4 *>(s_ent + kSplitWarps * kEntries);
  float *s_blk =
      reinterpret_cast<float *>(s_cache + kSplitWarps * kCellChunks * kCellSlots);
  const int nblk = (S + kSrcBlock - 1) / kSrcBlock;
  float *s_dh = s_blk + 2 * nblk;  // delta_hi of every source, contiguous
  int *s_tags = reinterpret_cast<int *>(s_dh + S);
  for (int i = threadIdx.x; i < kSplitWarps * kCellSlots; i += blockDim.x)
    s_tags[i] = -1;
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
  b.ent_base = s_ent;
  b.cell_cache = s_cache;
  b.cell_tags = s_tags;
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

// Work one warp performed (warp-uniform counts), for the launch statistics
struct SplitCounts {
  unsigned long long terms = 0;   // terms evaluated
  unsigned long long pairs = 0;   // (entry, source) pairs tested
  unsigned long long ivals = 0;   // lattice-point intervals solved
  unsigned long long blocks = 0;  // source blocks tested
};

// Per-warp queue of (entry, source) pairs: entries [e0, en) of the ring
// are pending, pairs [ch, ct) of the pixel's sequence are not yet summed.
struct PairQueue {
  int e0 = 0, en = 0, ch = 0, ct = 0;
};

// Appends one entry per lane with len > 0 (sources k1 .. k1 + len - 1 of the
// item whose state the lane holds; r and d4 as SplitEntry describes), in
// lane order.  Called by all lanes.
__device__ __forceinline__ void push_entries(
    SplitEntry *ring, PairQueue &pq, int len, int k1, int aux,
    const float Gh[3], const float r[3], const float Gl[3], const float rl[3],
    float4 d4) {
  const int lane = threadIdx.x & 31;
  const unsigned hm = __ballot_sync(0xffffffffu, len > 0);
  if (hm == 0u) return;
  int inc = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  const int tot = __shfl_sync(0xffffffffu, inc, 31);
  if (len > 0) {
    SplitEntry &E =
        ring[(pq.en + __popc(hm & ((1u << lane) - 1u))) & (kEntries - 1)];
    E.a = make_float4(Gh[0], Gh[1], r[0], r[1]);
    E.b = make_float4(Gl[0], Gl[1], rl[0], rl[1]);
    E.c = make_float4(Gh[2], r[2], Gl[2], rl[2]);
    E.d = d4;
    E.m = make_int4(k1, len, pq.ct + inc - len, aux);
  }
  pq.en += __popc(hm);
  pq.ct += tot;
  __syncwarp();
}

// Sums the next min(32, ct - ch) pairs of the queue, one per lane: the exact
// fractional offset of the step, the cut test, and for a surviving step its
// term (F_cell from the cell cache, F_latt, weight) into the lane's Kahan
// sum.  Called by all lanes; returns the number of surviving terms.
template <int INTERP, int HASDIV>
__device__ __forceinline__ unsigned sum_pairs(
    const SpotArgs &a, const SplitBlock &b, const SplitEntry *ring,
    PairQueue &pq, const float *unit, float4 *cache, int *tags, Kahan &acc) {
  const int lane = threadIdx.x & 31;
  const int np = min(32, pq.ct - pq.ch);
  // entries e0 .. e0 + 31 can overlap the window [ch, ch + 32)
  int4 mm = make_int4(0, 0, 0x7fffffff, 0);
  if (pq.e0 + lane < pq.en) mm = ring[(pq.e0 + lane) & (kEntries - 1)].m;
  const bool ov = pq.e0 + lane < pq.en && mm.z < pq.ch + np &&
                  mm.z + mm.y > pq.ch;
  // bit j of M: some entry starts at pair ch + j (entry e0 at bit 0)
  const unsigned M = __reduce_or_sync(
      0xffffffffu, ov ? 1u << max(mm.z - pq.ch, 0) : 0u);
  const int j = __popc(M & (0xffffffffu >> (31 - lane))) - 1;
  const int k1 = __shfl_sync(0xffffffffu, mm.x, j);
  const int pos = __shfl_sync(0xffffffffu, mm.z, j);
  const int aux = __shfl_sync(0xffffffffu, mm.w, j);
  const unsigned done =
      __ballot_sync(0xffffffffu, ov && mm.z + mm.y <= pq.ch + np);
  const bool valid = lane < np;
  const int k =
      valid ? (int)nb_idx(a.check, NB_SITE_SOURCE, k1 + (pq.ch + lane - pos),
                          b.S)
            : 0;
  const SplitEntry &E = ring[(pq.e0 + j) & (kEntries - 1)];
  const float4 A = E.a, B = E.b, C = E.c, D = E.d;
  const float Gh[3] = {A.x, A.y, C.x}, r[3] = {A.z, A.w, C.y};
  const float Gl[3] = {B.x, B.y, C.z}, rl[3] = {B.z, B.w, C.w};
  const float *src = b.src + k * SRC32_STRIDE;
  // (delta_lo, w, delta_hi) of source k in one load
  const float4 sw = *reinterpret_cast<const float4 *>(src);
  const float dh = sw.z;
  const float2 dlw = make_float2(sw.x, sw.y);
  float fr[3];
  int n[3];
  if (!HASDIV && (aux & kIntervalEntry)) {
    // G_hi d_hi + (r_q - (m - n0)) in one rounding plus the small terms;
    // the nearest integer is m
    // axes h and k in packed FMAs, l in scalar ones (the same roundings)
    const float2 dh2 = make_float2(dh, dh), dl2 = make_float2(dlw.x, dlw.x);
    const float2 f01 =
        fadd2(ffma2(make_float2(A.x, A.y), dh2, make_float2(A.z, A.w)),
              ffma2(make_float2(A.x, A.y), dl2,
                    ffma2(make_float2(B.x, B.y), dh2, make_float2(B.z, B.w))));
    fr[0] = f01.x;
    fr[1] = f01.y;
    fr[2] = fmaf(Gh[2], dh, r[2]) + fmaf(Gh[2], dlw.x, fmaf(Gl[2], dh, rl[2]));
    if (INTERP == 1 && a.C4) {
      // the packed index; unpacked only where a term needs the table
      // itself (term_value's fallback)
      n[0] = __float_as_int(D.y);
      n[1] = n[2] = kPackedIndex;
    } else {
      n[0] = __float_as_int(D.x);
      n[1] = __float_as_int(D.y);
      n[2] = __float_as_int(D.z);
    }
  } else {
    const float n0[3] = {D.x, D.y, D.z};
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      float tq = fmaf(Gh[x], dh, r[x]);
      float e0 = 0.f, e1 = 0.f;
      if (HASDIV) {
        const size_t e = ((size_t)(aux & 0xffff) * b.S + k) * 3 + x;
        e0 = __ldg(a.divh + e);
        e1 = __ldg(a.divl + e);
        tq -= e0;
      }
      float nf = rintf(tq);
      // G_hi d_hi + (r_q - n) in one rounding (r_q on a 2^-21 grid makes
      // r_q - n exact) plus the small terms
      const float sx = fmaf(Gh[x], dh, __fsub_rn(r[x], nf));
      const float c = fmaf(Gh[x], dlw.x, fmaf(Gl[x], dh, rl[x]));
      fr[x] = sx + c;
      if (HASDIV) {
        // the divergence term moves h after the rint: re-centre
        fr[x] -= e0 + e1;
        const float n2 = rintf(fr[x]);
        fr[x] -= n2;
        nf += n2;
      }
      n[x] = __float2int_rn(n0[x] + nf) - a.hmin[x];
    }
  }
  float rad2 = a.N[0] * a.N[0] * fr[0] * fr[0];
  rad2 = fmaf(a.N[1] * a.N[1], fr[1] * fr[1], rad2);
  rad2 = fmaf(a.N[2] * a.N[2], fr[2] * fr[2], rad2);
  const bool hit = valid && rad2 <= kGaussCut * 0.63f;
  float w = dlw.y * D.w;
  if (HASDIV && hit) {
    const float *df = unit + ((aux >> 16) & 31) * kUnitFloats + 7;
    const float *dir = src + SRC32_DIR, *ev = src + SRC32_E,
                *bv = src + SRC32_B;
    const float c2 = df[0] * dir[0] + df[1] * dir[1] + df[2] * dir[2];
    const float xx = df[0] * ev[0] + df[1] * ev[1] + df[2] * ev[2];
    const float yy = df[0] * bv[0] + df[1] * bv[1] + df[2] * bv[2];
    w *= 0.5f * (1.f + c2 * c2 - a.kahn * (xx * xx - yy * yy));
  }
  const unsigned hm = __ballot_sync(0xffffffffu, hit);
  if (hm != 0u) {
    CellRef cr;
    if (INTERP == 1 && !HASDIV && a.C4 && (aux & kIntervalEntry))
      cell_of_entry(a, hit, fr, __float_as_int(D.x), __float_as_int(D.z), cr);
    else
      cell_of<INTERP>(a, hit, fr, n, cr);
    const float t =
        term_value<INTERP>(a, hit, cr, fr, n, rad2, w, cache, tags);
    if (hit) acc.add(t);
  }
  pq.e0 += __popc(done);
  pq.ch += np;
  __syncwarp();  // the ring slots read above may be refilled next
  return __popc(hm);
}

// The sum, without the prefactor, of the pixel whose U sub-pixel units are
// already in `unit` (split_unit), computed by the calling warp (all 32
// lanes); every lane returns the same value.  Adds the terms it evaluated
// to `cnt` and, with COUNT, the rest of the work it performed.
template <int INTERP, int HASDIV, int COUNT = 0>
__device__ __forceinline__ double split_sum(const SpotArgs &a,
                                            const SplitBlock &b,
                                            const float *unit,
                                            SplitCounts &cnt) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int PM = b.PM, S = b.S, nblk = b.nblk, sstep = b.sstep;
  const float2 *s_ax2 = b.ax2;
  const float *s_blk = b.blk, *s_dh = b.dh;
  SplitEntry *ring = b.ent_base + warp * kEntries;
  float4 *cache = b.cell_cache + warp * kCellChunks * kCellSlots;
  int *tags = b.cell_tags + warp * kCellSlots;
  const int U = a.os * a.os * a.T, items = U * PM;
  const float N2[3] = {a.N[0] * a.N[0], a.N[1] * a.N[1], a.N[2] * a.N[2]};
  const float cwide = b.cwide;
  const float cmarg[3] = {b.cmarg[0], b.cmarg[1], b.cmarg[2]};
  const bool iv_ok = b.iv_ok;
  const float dmin = b.dmin, dmax = b.dmax, dmarg = b.dmarg;
  const bool even = b.even;
  const float inv_step = b.inv_step;
  const float u0h = b.u0h, u0l = b.u0l;

  Kahan acc;
  PairQueue pq;
  unsigned nterms = 0, nivals = 0, nblocks = 0;
  auto drain = [&]() {
    while (pq.ct - pq.ch >= 32)
      nterms += sum_pairs<INTERP, HASDIV>(a, b, ring, pq, unit, cache, tags,
                                          acc);
  };
  // ---- items: lanes take (unit, phi x mosaic) items 32 at a time, form
  // G and r, and push their source intervals; the pair queue is summed
  // 32 pairs at a time as it fills
  for (int base = 0; base < items; base += 32) {
    const int it = base + lane;
    const bool valid = it < items;
    const int u = valid ? it / PM : 0, pm = valid ? it - u * PM : 0;
    const float *ud = unit + u * kUnitFloats;
    // vh[3], vl[3], scal as four float2 loads (unit rows are 8-byte aligned)
    const float2 *u2 = reinterpret_cast<const float2 *>(ud);
    const float2 p0 = u2[0], p1 = u2[1], p2 = u2[2], p3 = u2[3];
    const float vh[3] = {p0.x, p0.y, p1.x}, vl[3] = {p1.y, p2.x, p2.y};
    const float scal = p3.x;
    float Gh[3], Gl[3], rq[3], rl[3], n0[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      ff_dot3_pairs(s_ax2 + pm * 9 + 3 * x, vh, vl, Gh[x], Gl[x]);
      float qh, qe;
      two_prod(Gh[x], u0h, qh, qe);
      const float ql = fmaf(Gh[x], u0l, fmaf(Gl[x], u0h, qe));
      n0[x] = rintf(qh);
      float rh, rl0;
      two_sum(__fsub_rn(qh, n0[x]), ql, rh, rl0);
      // r_hi on a 2^-21 grid: r_hi - n is then exact for |n| < 7
      rq[x] = __fmul_rn(rintf(__fmul_rn(rh, 2097152.f)), 1.f / 2097152.f);
      rl[x] = rl0 + __fsub_rn(rh, rq[x]);
    }
    if (HASDIV) {
      // sources of different directions: every source of every item
      push_entries(ring, pq, valid ? S : 0, 0, pm | (u << 16), Gh, rq, Gl, rl,
                   make_float4(n0[0], n0[1], n0[2], scal));
      drain();
      continue;
    }
    // lattice points the item's sweep can come near: per axis the
    // integers within sqrt(cwide)/N_x of [h(dmin), h(dmax)]
    int ml[3] = {0, 0, 0}, nm[3] = {0, 0, 0}, ncomb = 0;
    if (iv_ok && valid) {
      ncomb = 1;
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const float lo = fmaf(Gh[x], dmin, rq[x]), hi = fmaf(Gh[x], dmax, rq[x]);
        ml[x] = (int)ceilf(fminf(lo, hi) - cmarg[x]);
        nm[x] = (int)floorf(fmaxf(lo, hi) + cmarg[x]) - ml[x] + 1;
        if (nm[x] < 0) nm[x] = 0;
        ncomb *= nm[x];
      }
    }
    if (iv_ok && __all_sync(0xffffffffu, ncomb <= 8)) {
      // exact intervals: for lattice point m the exponent sum along the
      // sweep is A d^2 + 2 B d + C, below cwide on one interval of the
      // sorted delta table
      const int maxc = (int)__reduce_max_sync(0xffffffffu, (unsigned)ncomb);
      if (COUNT) nivals += __reduce_add_sync(0xffffffffu, (unsigned)ncomb);
      // the lattice points ml + (d0, d1, d2), d_x < nm_x, in odometer order;
      // A of the quadratic depends on the item only
      float A = N2[0] * Gh[0] * Gh[0];
      A = fmaf(N2[1] * Gh[1], Gh[1], A);
      A = fmaf(N2[2] * Gh[2], Gh[2], A);
      int dg[3] = {0, 0, 0};
      for (int c = 0; c < maxc; ++c) {
        int k1 = 0, k2 = 0;
        float dx[3] = {0.f, 0.f, 0.f};
        int nt[3] = {0, 0, 0};
        if (c < ncomb) {
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            // lattice point n0 + mx; its table index nt
            const int mx = ml[x] + dg[x];
            dx[x] = rq[x] - (float)mx;  // exact: r_q on a 2^-21 grid
            nt[x] = (int)n0[x] + mx - a.hmin[x];
          }
          if (++dg[0] == nm[0]) {
            dg[0] = 0;
            if (++dg[1] == nm[1]) {
              dg[1] = 0;
              ++dg[2];
            }
          }
          float B = N2[0] * Gh[0] * dx[0];
          B = fmaf(N2[1] * Gh[1], dx[1], B);
          B = fmaf(N2[2] * Gh[2], dx[2], B);
          float C0 = N2[0] * dx[0] * dx[0];
          C0 = fmaf(N2[1] * dx[1], dx[1], C0);
          C0 = fmaf(N2[2] * dx[2], dx[2], C0);
          if (A > 0.f) {
            const float disc = fmaf(B, B, -A * (C0 - cwide));
            if (disc >= 0.f) {
              // the bounds carry a relative margin far above the error of
              // the reciprocal
              const float sq = sqrtf(disc), ia = __frcp_rn(A);
              float lo = (-B - sq) * ia, hi = (-B + sq) * ia;
              const float mg = 1e-4f * (fabsf(lo) + fabsf(hi)) + dmarg;
              lo -= mg;
              hi += mg;
              // k1 = #{delta < lo}, k2 = #{delta <= hi} (sorted table)
              if (even) {
                k1 = count_below(s_dh, S, guess_index(lo, dmin, inv_step, S),
                                 lo);
                k2 = count_at_most(s_dh, S, guess_index(hi, dmin, inv_step, S),
                                   hi);
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
        // no lane has an entry for this lattice point: nothing to push
        if (!__any_sync(0xffffffffu, k2 > k1)) continue;
        float4 d4;
        if (INTERP == 1 && a.C4) {
          // the lattice point's cell data once per entry; the index packed
          // (clamped to [-1, hn]: any index outside the table looks up
          // default_F, and cell tables exist only for hn < 1024)
          int ci0 = 0, pk = 0, npk = 0;
          if (k2 > k1) {
            entry_cell_data(a, nt, ci0, pk);
#pragma unroll
            for (int x = 0; x < 3; ++x)
              npk |= (min(max(nt[x], -1), a.hn[x]) + 1) << (10 * x);
          }
          d4 = make_float4(__int_as_float(ci0), __int_as_float(npk),
                           __int_as_float(pk), scal);
        } else {
          d4 = make_float4(__int_as_float(nt[0]), __int_as_float(nt[1]),
                           __int_as_float(nt[2]), scal);
        }
        push_entries(ring, pq, k2 > k1 ? k2 - k1 : 0, k1,
                     pm | (u << 16) | kIntervalEntry, Gh, dx, Gl, rl, d4);
        drain();
      }
    } else {
      // pruned scan: h_x = G_x delta + r_x is linear in delta, so a block
      // of sources whose delta range [dmn, dmx] keeps some axis farther
      // than sqrt(cut)/N_x from every integer holds no surviving term
      if (COUNT) nblocks += __popc(__ballot_sync(0xffffffffu, valid)) * nblk;
      for (int bb = 0; bb < nblk; ++bb) {
        bool pass = false;
        if (valid) {
          const float dmn = s_blk[2 * bb], dmx = s_blk[2 * bb + 1];
          pass = true;
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            const float lo0 = fmaf(Gh[x], dmn, rq[x]),
                        hi0 = fmaf(Gh[x], dmx, rq[x]);
            const float lo = fminf(lo0, hi0) - cmarg[x],
                        hi = fmaxf(lo0, hi0) + cmarg[x];
            pass = pass && floorf(hi) >= ceilf(lo);
          }
        }
        const int st0 = bb * kSrcBlock;
        push_entries(ring, pq, pass ? min(kSrcBlock, S - st0) : 0, st0,
                     pm | (u << 16), Gh, rq, Gl, rl,
                     make_float4(n0[0], n0[1], n0[2], scal));
        drain();
      }
    }
  }
  if (pq.ct > pq.ch)
    nterms += sum_pairs<INTERP, HASDIV>(a, b, ring, pq, unit, cache, tags, acc);
  cnt.terms += nterms;
  if (COUNT) {
    cnt.pairs += pq.ct;
    cnt.ivals += nivals;
    cnt.blocks += nblocks;
  }

  // ---- warp reduction in float-float: each lane's compensated sum is
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
