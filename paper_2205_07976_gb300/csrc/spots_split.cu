// spots_split.cu -- the FP32-mixed Bragg-spot sum for Gaussian lattice
// shapes, one warp per pixel (the per-pixel step reduction of Sec. III-B's
// nanoBraggSpots, split across lanes, with the fused addArray accumulate).
//
// Why a second variant: with a Gaussian F_latt only a few percent of the
// (subpixel, layer, phi x mosaic, source) steps of a pixel carry a term that
// does not underflow in FP32, and each such term needs the structure factor
// (64 gathers for tricubic interpolation).  With one thread per pixel those
// terms are scattered over lanes and a warp serialises them.  Here:
//   1. a warp takes B = 32 / U pixels at a time (one when it gets fewer
//      than 256 pixels in all); its lanes set up the
//      U = os^2 x layers sub-pixel units of all B pixels in FP64 (position,
//      direction, solid angle, capture, polarization) into shared memory,
//      then the warp sums the pixels one after another;
//   2. lanes take (unit, phi x mosaic) items 32 at a time and form G and r
//      in double-float.  h_x = G_x delta + r_x is linear in a source's
//      delta = 1/lambda - u0, so for each lattice point near the item's
//      sweep the sources whose exponent sum N^2 f^2 / 0.63 can stay below
//      the underflow cut form one interval of the sorted delta table (a
//      quadratic in delta, then a short search); where that does not
//      apply, blocks of 8 sources are pruned by their delta range.  Each
//      non-empty interval becomes one entry of a per-warp ring in shared
//      memory, holding a copy of its item's state;
//   3. whenever the ring holds 32 (entry, source) pairs, each lane takes
//      one pair, forms the step's exact fractional offset and, if the step
//      survives the cut, its term (exp, F_cell from the cell's tricubic
//      polynomial in a per-warp shared-memory cache, or from the table)
//      into its own Kahan sum;
//   4. the 32 lane sums are reduced with warp shuffles in float-float.
// The order of every operation depends only on the pixel's own inputs, so
// a pixel's value does not depend on what else is in the launch.
// Pixels are handed to warps through an atomic counter in a scratch word.
#include "split_pixel.cuh"

namespace nbgb {

// COUNT: also count the pairs, intervals and block tests (a.wstats)
template <int INTERP, int HASDIV, int COUNT>
__global__ void __launch_bounds__(kSplitThreads, 5)
    spots_split_kernel(SpotArgs a, unsigned long long *work) {
  extern __shared__ float sms[];
  SplitBlock b;
  split_stage(b, sms, a, a.axh, a.axl, a.src32, a.PM, a.S, a.u0h, a.u0l);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long n_work = a.pixlist ? a.n_list : a.npix;
  SplitCounts cnt;  // work of this warp
  // a warp takes B pixels at a time and sets up all their sub-pixel units
  // in one pass, so the FP64 geometry fills up to 32 lanes
  // (one pixel at a time when a warp gets few pixels: pixels differ in
  // cost, and grabbing several near the end of a launch leaves a tail)
  const int U = a.os * a.os * a.T;
  const long long per_warp = n_work / ((long long)gridDim.x * kSplitWarps);
  const int B = per_warp >= 256 ? kMaxUnits / U : 1;
  float *unit = b.unit_base + warp * kMaxUnits * kUnitFloats;
  while (true) {
    long long first = 0;
    if (lane == 0) first = (long long)atomicAdd(work, (unsigned long long)B);
    first = __shfl_sync(0xffffffffu, first, 0);
    if (first >= n_work) break;
    const int nb = (int)min((long long)B, n_work - first);
    if (lane < nb * U) {
      const int bi = lane / U;
      const long long gp = a.pixlist ? a.pixlist[first + bi] : first + bi;
      const DevPanel &P = a.panels[panel_of_pixel(a, gp)];
      const long long local = gp - P.pix0;
      const int s = (int)(local / P.nfast);
      const int f = (int)(local - (long long)s * P.nfast);
      split_unit<HASDIV>(a, P, s, f, lane - bi * U, unit + lane * kUnitFloats);
    }
    __syncwarp();
    double mine = 0.0;  // lane bi keeps the sum of pixel bi
    for (int bi = 0; bi < nb; ++bi) {
      const double v = split_sum<INTERP, HASDIV, COUNT>(
          a, b, unit + bi * U * kUnitFloats, cnt);
      if (lane == bi) mine = v;
    }
    // fused accumulate into the image: lanes 0 .. nb-1 add the batch's
    // pixels, consecutive in the image, in one coalesced access
    if (lane < nb) {
      const long long gp = a.pixlist ? a.pixlist[first + lane] : first + lane;
      a.image[nb_idx(a.check, NB_SITE_IMAGE, gp, a.npix)] +=
          a.prefactor * mine;
    }
    __syncwarp();  // the next batch rewrites the units
  }
  if (lane == 0 && a.stats && cnt.terms) atomicAdd(a.stats, cnt.terms);
  if (COUNT && lane == 0 && a.wstats) {
    atomicAdd(a.wstats, cnt.pairs);
    atomicAdd(a.wstats + 1, cnt.ivals);
    atomicAdd(a.wstats + 2, cnt.blocks);
  }
}

size_t split_smem_bytes(const SpotArgs &a) {
  return split_smem_layout(a.PM, a.S);
}

bool split_supported(const SpotArgs &a) {
  return a.shape == 1 && a.os * a.os * a.T <= kMaxUnits &&
         split_smem_bytes(a) <= 200 * 1024;
}

cudaError_t launch_spots_split(const SpotArgs &a, unsigned long long *work,
                               int sm_count, cudaStream_t st) {
  size_t smem = split_smem_bytes(a);
  void (*kern)(SpotArgs, unsigned long long *);
  if (a.wstats)
    kern = a.interp ? (a.has_div ? spots_split_kernel<1, 1, 1>
                                 : spots_split_kernel<1, 0, 1>)
                    : (a.has_div ? spots_split_kernel<0, 1, 1>
                                 : spots_split_kernel<0, 0, 1>);
  else
    kern = a.interp ? (a.has_div ? spots_split_kernel<1, 1, 0>
                                 : spots_split_kernel<1, 0, 0>)
                    : (a.has_div ? spots_split_kernel<0, 1, 0>
                                 : spots_split_kernel<0, 0, 0>);
  cudaError_t e = cudaFuncSetAttribute(
      kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern,
                                                    kSplitThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  long long n_work = a.pixlist ? a.n_list : a.npix;
  long long blocks = (long long)sm_count * per_sm;
  long long need = (n_work + kSplitWarps - 1) / kSplitWarps;
  if (blocks > need) blocks = need;
  if (blocks < 1) return cudaSuccess;
  kern<<<(unsigned)blocks, kSplitThreads, smem, st>>>(a, work);
  return cudaGetLastError();
}

}  // namespace nbgb
