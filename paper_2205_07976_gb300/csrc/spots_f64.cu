// spots_f64.cu -- the plain FP64 form of the per-pixel Bragg-spot sum
// (nanoBraggSpots, Sec. III-B), one thread per pixel, with the fused
// double accumulate of addArray (Listing 1).
//
// Loop nest per pixel: subpixel x sensor layer -> source -> phi x mosaic.
// Everything is FP64 and this file is compiled without FMA contraction.
// The Miller indices, the fractional offsets and the sinc are evaluated in
// the order the definition is written, so h and the sinc's phases are
// bitwise those of any other uncontracted FP64 evaluation (the sinc at
// N = 200 multiplies h's rounding by pi N).  The rest, which is not
// sensitive to the last bits, is arranged for the FP64 pipe, which on this
// part issues at 1/64 of the FP32 rate and so sets the kernel's time:
//   * the sinc's denominators sin(pi f), |pi f| <= pi/2, come from a
//     truncated Taylor series (sin_half_period) instead of the general
//     sine with its range reduction; their argument is unchanged;
//   * the Gaussian exponent (summed in explicit FMAs) and the Lagrange
//     weights multiply by 1/0.63 and 1/6 instead of dividing, and the sinc
//     divides once per step, not once per axis (an IEEE division is a
//     sequence of about ten FP64 instructions; the result moves by an ulp
//     or two);
//   * the tricubic sum is nested per axis in explicit FMAs, sum_i w_i
//     sum_j w_j sum_k w_k F_ijk: 84 FP64 operations instead of 256 for the
//     flat triple product sum (the rounding differs at the 1e-15 level);
//   * the table is read from an FP64 copy (a float-to-double conversion
//     is an FP64-pipe instruction too), and the cell's first node comes
//     from the nearest lattice point instead of a floor;
//   * the step's weight, capture, polarization and solid angle are one
//     factor per source.
// Only loop invariants are hoisted (pixel position, solid angle, capture
// fraction per subpixel/layer; scattering vector, polarization and that
// factor per source).  The rotated axes and the source table are staged in
// shared memory per block.
#include "nbgb_internal.cuh"

namespace nbgb {

__device__ __forceinline__ double dot3d(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// sin(x) for |x| <= pi/2 from its Taylor series through x^21/21!: the
// remainder is below (pi/2)^23/23! < 2e-18, the coefficients are the
// reciprocal factorials rounded once (every factorial up to 21! is exact
// in FP64), and x + x^3 p with p by Horner in x^2 keeps the error to a few
// ulp; 12 FP64 operations, no range reduction (the sinc's denominators
// have |pi f| <= pi/2)
__device__ __forceinline__ double sin_half_period(double x) {
  const double x2 = x * x;
  double p = 1.0 / 51090942171709440000.0;  // 1/21!
  p = fma(p, x2, -1.0 / 121645100408832000.0);
  p = fma(p, x2, 1.0 / 355687428096000.0);
  p = fma(p, x2, -1.0 / 1307674368000.0);
  p = fma(p, x2, 1.0 / 6227020800.0);
  p = fma(p, x2, -1.0 / 39916800.0);
  p = fma(p, x2, 1.0 / 362880.0);
  p = fma(p, x2, -1.0 / 5040.0);
  p = fma(p, x2, 1.0 / 120.0);
  p = fma(p, x2, -1.0 / 6.0);
  return fma(x * x2, p, x);
}

template <int SHAPE>
__device__ __forceinline__ double flatt_f64(const SpotArgs &a,
                                            const double h[3], double n[3]) {
  // sinc: the three numerators and the three denominators multiplied
  // separately and divided once (a division is a sequence of about ten
  // FP64 instructions); an axis with |f| below 1e-100 (f = 0 in practice:
  // h is a sum of products of order-one values) contributes its limit N,
  // so the product of denominators cannot underflow
  double num = 1.0, den = 1.0, rad2 = 0.0;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    n[x] = ceil(h[x] - 0.5);  // nearest integer, ties down
    double fr = h[x] - n[x];
    if (SHAPE == 0) {
      // sin(pi N h)/sin(pi h) = +-sin(pi N f)/sin(pi f); the sign drops out
      // |f| < 1e-100 as an integer compare of the magnitudes' bit patterns
      // (ordered like the values for non-negative doubles; a double
      // compare is one more FP64-pipe instruction)
      if ((__double_as_longlong(fr) & 0x7fffffffffffffffll) <
          __double_as_longlong(1e-100)) {
        num *= a.N64[x];
      } else {
        num *= sin(M_PI * a.N64[x] * fr);
        den *= sin_half_period(M_PI * fr);
      }
    } else {
      // sum N^2 f^2 / 0.63 in explicit FMAs (N^2 / 0.63 is loop-invariant)
      rad2 = fma(a.N64[x] * a.N64[x] * (1.0 / 0.63) * fr, fr, rad2);
    }
  }
  if (SHAPE == 1) return a.N64[0] * a.N64[1] * a.N64[2] * exp(-rad2);
  return num / den;
}

__device__ __forceinline__ bool in_table(const SpotArgs &a, long long i,
                                         long long j, long long k) {
  return (unsigned long long)i < (unsigned long long)a.hn[0] &&
         (unsigned long long)j < (unsigned long long)a.hn[1] &&
         (unsigned long long)k < (unsigned long long)a.hn[2];
}

// The tricubic sum over the 4x4x4 stencil whose first node has flat index
// off: nested per axis in explicit FMAs, sum_i w_i sum_j w_j sum_k w_k
// F_ijk (84 FP64 operations; a flat triple-product sum takes 256).  T is
// double (the FP64 copy of the table) or float (each read converted).
template <typename T>
__device__ __forceinline__ double tricubic_sum(const SpotArgs &a,
                                               const T *tab, long long off,
                                               const double w[3][4]) {
  double sum = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double si = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T *row = tab + off + ((long long)i * a.hn[1] + j) * a.hn[2];
      double sj = w[2][0] * (double)__ldg(row);
      sj = fma(w[2][1], (double)__ldg(row + 1), sj);
      sj = fma(w[2][2], (double)__ldg(row + 2), sj);
      sj = fma(w[2][3], (double)__ldg(row + 3), sj);
      si = j ? fma(w[1][j], sj, si) : w[1][0] * sj;
    }
    sum = i ? fma(w[0][i], si, sum) : w[0][0] * si;
  }
  return sum;
}

// F_cell at h, whose nearest lattice point is n (ties down, flatt_f64):
// the cell's first node is floor(h) = n - 1 where h < n, else n, so no
// floor and no second float-to-integer conversion per axis are needed
template <int INTERP>
__device__ __forceinline__ double fcell_f64(const SpotArgs &a,
                                            const double h[3],
                                            const double n[3]) {
  long long nn[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) nn[c] = (long long)n[c] - a.hmin[c];
  if (INTERP == 1) {
    long long fl[3];
    double x[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // h - n is exact (h and n lie within 1/2), and so is h - floor(h)
      // for h < n: (h - n) + 1 holds no bit below h's last one
      const double fr = h[c] - n[c];
      // f < 0 from the sign bit (an integer test; f = h - n is never -0)
      const bool below = __double_as_longlong(fr) < 0;
      fl[c] = nn[c] - (below ? 1 : 0);
      x[c] = below ? fr + 1.0 : fr;
    }
    if (in_table(a, fl[0] - 1, fl[1] - 1, fl[2] - 1) &&
        in_table(a, fl[0] + 2, fl[1] + 2, fl[2] + 2)) {
      // 4-point Lagrange weights on nodes -1, 0, 1, 2, from the shared
      // products t (t - 1) / 6 and (t + 1)(t - 2) / 2 (11 operations per
      // axis; the negations are free operand modifiers)
      double w[3][4];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double t = x[c], tm1 = t - 1.0, tm2 = t - 2.0, tp1 = t + 1.0;
        const double p6 = t * tm1 * (1.0 / 6.0), q2 = tp1 * tm2 * 0.5;
        w[c][0] = -(p6 * tm2);
        w[c][1] = q2 * tm1;
        w[c][2] = -(q2 * t);
        w[c][3] = p6 * tp1;
      }
      long long off =
          ((long long)(fl[0] - 1) * a.hn[1] + (fl[1] - 1)) * a.hn[2] +
          (fl[2] - 1);
      {
        const long long last = off + (3ll * a.hn[1] + 3) * a.hn[2] + 3;
        if (nb_idx(a.check, NB_SITE_STENCIL, last, table_size(a)) != last)
          off = 0;
      }
      return a.F64t ? tricubic_sum(a, a.F64t, off, w)
                    : tricubic_sum(a, a.F, off, w);
    }
  }
  if (in_table(a, nn[0], nn[1], nn[2])) {
    const long long idx = nb_idx(a.check, NB_SITE_F,
                                 (nn[0] * a.hn[1] + nn[1]) * a.hn[2] + nn[2],
                                 table_size(a));
    return a.F64t ? __ldg(a.F64t + idx) : (double)__ldg(a.F + idx);
  }
  return a.defF64;
}

// F as doubles, for the NB_F64 kernel's reads
__global__ void f64_table_kernel(const float *F, long long n, double *F64t) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    F64t[i] = (double)F[i];
}

cudaError_t build_f64_table(const float *F, long long n, double *F64t,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  f64_table_kernel<<<1216, 256, 0, st>>>(F, n, F64t);
  return cudaGetLastError();
}

template <int SHAPE, int INTERP>
__global__ void __launch_bounds__(kTileThreads, 4)
    spots_f64_kernel(SpotArgs a) {
  extern __shared__ double sm[];
  double *s_ax = sm;
  double *s_src = sm + a.PM * 9;
  for (int i = threadIdx.x; i < a.PM * 9; i += blockDim.x) s_ax[i] = a.ax64[i];
  for (int i = threadIdx.x; i < a.S * SRC64_STRIDE; i += blockDim.x)
    s_src[i] = a.src64[i];
  __syncthreads();

  long long item = a.pixlist ? (long long)blockIdx.x * blockDim.x + threadIdx.x
                             : (long long)blockIdx.x;
  long long gp;
  int q, s, f;
  if (!map_pixel(a, item, threadIdx.x, gp, q, s, f)) return;
  const DevPanel &P = a.panels[q];
  const double px = P.px;
  const int os = a.os;
  double acc = 0.0;
  for (int i = 0; i < os; ++i) {
    for (int j = 0; j < os; ++j) {
      for (int t = 0; t < a.T; ++t) {
        double cf = (f + (i + 0.5) / os) * px, cs = (s + (j + 0.5) / os) * px,
               cn = t * a.dt;
        double pos[3], d[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          pos[c] = P.origin[c] + cf * P.fdir[c] + cs * P.sdir[c] +
                   cn * P.ndir[c];
        double R = sqrt(dot3d(pos, pos));
#pragma unroll
        for (int c = 0; c < 3; ++c) d[c] = pos[c] / R;
        double omega = px * px * dot3d(P.ndir, pos) / (R * R * R);
        double cap = 1.0;
        if (a.thickness > 0.0) {
          double L = a.atten * dot3d(d, P.ndir);
          cap = exp(-t * a.dt / L) - exp(-(t + 1) * a.dt / L);
        }
        for (int k = 0; k < a.S; ++k) {
          const double *src = s_src + k * SRC64_STRIDE;
          const double lam = src[SRC64_LAM];
          const double *dir = src + SRC64_DIR;
          double Sv[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) Sv[c] = (d[c] - dir[c]) / lam;
          // Kahn: cos 2psi sin^2 2theta = (d.E')^2 - (d.B')^2 for unit d
          double c2 = dot3d(d, dir), x = dot3d(d, src + SRC64_E),
                 y = dot3d(d, src + SRC64_B);
          double pol = 0.5 * (1.0 + c2 * c2 - a.kahn64 * (x * x - y * y));
          // the step's factors that do not depend on phi x mosaic
          const double wcpo = src[SRC64_W] * cap * pol * omega;
          for (int pm = 0; pm < a.PM; ++pm) {
            const double *A = s_ax + pm * 9;
            double h[3] = {dot3d(A, Sv), dot3d(A + 3, Sv), dot3d(A + 6, Sv)};
            double n[3];
            double fl = flatt_f64<SHAPE>(a, h, n);
            double fc = fcell_f64<INTERP>(a, h, n);
            const double a_ = fc * fl;
            acc += a_ * a_ * wcpo;
          }
        }
      }
    }
  }
  a.image[nb_idx(a.check, NB_SITE_IMAGE, gp, a.npix)] += a.prefactor * acc;
}

cudaError_t launch_spots_f64(const SpotArgs &a, cudaStream_t st) {
  size_t smem = (size_t)(a.PM * 9 + a.S * SRC64_STRIDE) * sizeof(double);
  long long blocks = a.pixlist ? (a.n_list + kTileThreads - 1) / kTileThreads
                               : a.n_tiles;
  if (blocks <= 0) return cudaSuccess;
  void (*kern)(SpotArgs) = nullptr;
  int key = a.shape * 2 + a.interp;
  switch (key) {
    case 0: kern = spots_f64_kernel<0, 0>; break;
    case 1: kern = spots_f64_kernel<0, 1>; break;
    case 2: kern = spots_f64_kernel<1, 0>; break;
    default: kern = spots_f64_kernel<1, 1>; break;
  }
  cudaError_t e = cudaFuncSetAttribute(
      kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)blocks, kTileThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace nbgb
