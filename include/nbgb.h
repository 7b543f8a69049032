/*
 * nbgb.h -- C ABI of the GB300 Bragg-spot library (libnbgb.so).
 *
 * The library computes the per-pixel Bragg-spot image of one crystal shot:
 * the nanoBraggSpots sum of Sec. III-B (every detector pixel independent;
 * the sum runs over crystal orientation, mosaic domains and photon energy,
 * with one structure factor per Bragg spot, Sec. II), here over
 * subpixels x sensor layers x sources x phi steps x mosaic domains:
 *
 *   I_p += r_e^2 fluence scale / (os^2 M Phi)
 *          * sum_{sub, layer, k, phi, m} F_cell(hkl)^2 F_latt(hkl)^2
 *                                       * w_k cap pol omega,
 *   hkl = (a, b, c)_{phi,m} . (d - i_k) / lambda_k,
 *   (a, b, c)_{phi,m} = U_m R_phi (a, b, c)_lab.
 *
 * and accumulates it into a resident double image, the fused form of the
 * addArray kernel of Sec. III-B (Listing 1: lhs[j] += (double) rhs[j]).
 *
 * Conventions
 *   - Every function returns an nb_status and never aborts or throws.
 *   - Every host array argument is copied before the call returns; the
 *     caller keeps ownership.  Device tables and the image belong to the
 *     handle until nb_free().
 *   - Lengths: Angstrom for crystal axes and wavelengths, metres for the
 *     detector.  The sample is at the origin.
 *   - Global pixel index: panel-major, then slow, then fast.
 *   - Work is queued on the handle's CUDA stream; nb_get_image() waits for it.
 *   - Calls on one handle must not overlap (one host thread at a time).
 */
#ifndef NBGB_H
#define NBGB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nb_sim nb_sim; /* opaque, owned by the library */

typedef enum {
    NB_OK = 0,
    NB_EINVAL = -1,   /* a bad argument (size, pointer, value)          */
    NB_ENOMEM = -2,   /* a device or host allocation failed             */
    NB_ECUDA = -3,    /* a CUDA call failed; nb_last_error() has text   */
    NB_ESTATE = -4,   /* called out of order (e.g. spots before setup)  */
    NB_ETIMEOUT = -5  /* a bounded device-side wait ran out             */
} nb_status;

typedef enum {
    NB_F64 = 0,   /* plain FP64 throughout                                  */
    NB_MIXED = 1, /* FP32 bulk; double-float scattering-vector.axis dots and
                     fractional offsets; compensated FP32 accumulation     */
    NB_F32 = 2    /* everything in FP32 (the precision sweep's lower arm)   */
} nb_precision;

enum { NB_SHAPE_SINC = 0, NB_SHAPE_GAUSS = 1 };
enum { NB_INTERP_NEAREST = 0, NB_INTERP_TRICUBIC = 1 };
enum { NB_DTYPE_F32 = 0, NB_DTYPE_F64 = 1 };

/* One flat detector panel.  Pixel (s, f), subpixel (i, j) of an oversample
 * os sits at origin + (f + (i+1/2)/os) pixel fdir + (s + (j+1/2)/os) pixel
 * sdir; sensor layer t adds t * thickness / n_layers * ndir. */
typedef struct {
    double origin[3]; /* m, outer corner of pixel (0, 0)                  */
    double fdir[3];   /* unit fast axis                                   */
    double sdir[3];   /* unit slow axis                                   */
    double ndir[3];   /* unit normal pointing away from the sample        */
    double pixel_m;   /* square pixel size, m                             */
    int nfast;
    int nslow;
} nb_panel;

/* Create a handle on CUDA device `device` computing in `precision`, with
 * its work queued on `cuda_stream` (a cudaStream_t; NULL: the legacy
 * default stream).  *out receives the handle; on failure *out is NULL.
 * Errors: NB_EINVAL (out NULL, bad precision), NB_ECUDA (bad device). */
int nb_sim_create(nb_sim **out, int device, int precision, void *cuda_stream);

/* Crystal (Sec. III-B: orientation and mosaicity; Sec. II: one structure
 * factor per spot).
 *   axes      9 doubles, rows a, b, c (Angstrom), lab frame, orientation
 *             included.
 *   umats     n_mosaic 3x3 row-major rotations U_m (mosaic domains).
 *   n_phi, phi0_deg, phistep_deg, spindle
 *             phi step j rotates the axes by phi0 + j*phistep degrees about
 *             the spindle (any non-zero vector) before U_m applies.
 *   Na, Nb, Nc  unit cells per mosaic block; integers for NB_SHAPE_SINC.
 *   shape     NB_SHAPE_SINC: F_latt = prod sin(pi N h)/sin(pi h);
 *             NB_SHAPE_GAUSS: F_latt = Na Nb Nc exp(-sum N^2 (h-h0)^2/0.63).
 *   F         structure-factor amplitudes, float, hkl_n[0] x hkl_n[1] x
 *             hkl_n[2], l fastest, for h in [hkl_min[0], hkl_min[0] +
 *             hkl_n[0]) and so on.  NULL keeps the table of the previous
 *             call (hkl_min, hkl_n, interp and default_F must then match or
 *             are ignored when they are NULL / negative).
 *   interp    NB_INTERP_NEAREST (F at the nearest node, default_F outside
 *             the table) or NB_INTERP_TRICUBIC (4-point Lagrange per axis;
 *             nearest where the 4x4x4 stencil leaves the table).
 * The table is copied to the device.  The first launch after a new table
 * derives from it what its kernels read: for NB_F64 a copy in doubles (2x
 * the table's memory), for the FP32 forms with tricubic lookup 16-byte
 * stencil rows (4x) and, for NB_MIXED's warp-per-pixel kernel and
 * adjoint, each cell's 64 polynomial coefficients (256 bytes per cell; not
 * built above 2 GB or 1000 nodes per axis); where one of these is not
 * built or its allocation fails, the kernels read F itself.
 * Errors: NB_EINVAL for n_mosaic < 1, n_phi < 1, n_mosaic x n_phi >
 * 2048, non-positive or (sinc) non-integral N, a zero spindle with
 * n_phi > 1, empty table, NULL axes or umats, or F NULL before any table
 * was set. */
int nb_set_crystal(nb_sim *sim, const double axes[9], const double *umats,
                   int n_mosaic, int n_phi, double phi0_deg,
                   double phistep_deg, const double spindle[3], double Na,
                   double Nb, double Nc, int shape, const float *F,
                   const int hkl_min[3], const int hkl_n[3], int interp,
                   double default_F);

/* Overall intensity scale of the crystal (default 1). */
int nb_set_scale(nb_sim *sim, double scale);

/* Beam (Sec. III-B: photon energy; Sec. II: shot-to-shot spectrum).
 *   dirs      n_src x 3 unit propagation directions.
 *   lambda_A  n_src wavelengths (Angstrom, > 0).
 *   weights   n_src weights w_k, used as given (pass weights summing to 1
 *             for `fluence` to be the total fluence).
 *   fluence   photons per m^2.
 *   kahn_K    polarization factor K in [0, 1]; e_vec the E-vector of the
 *             polarized part (not parallel to any source direction when
 *             K != 0).
 * The library keeps the sources ordered by ascending 1/lambda (the sum does
 * not depend on their order; results agree to rounding).
 * Errors: NB_EINVAL for n_src outside [1, 1024], NULL arrays, non-unit
 * directions, lambda <= 0, K outside [0, 1], or e_vec parallel to a
 * direction. */
int nb_set_beam(nb_sim *sim, const double *dirs, const double *lambda_A,
                const double *weights, int n_src, double fluence,
                double kahn_K, const double e_vec[3]);

/* Detector: n_panels panels (copied), oversample os >= 1 per axis,
 * n_layers >= 1 sensor layers of a sensor `thickness_m` thick with
 * attenuation length `atten_m`.  thickness 0 means a surface detector (the
 * capture fraction is 1; n_layers must then be 1).  Resets the image to 0.
 * Errors: NB_EINVAL for empty panels, non-positive sizes, layers with no
 * thickness, atten_m <= 0 with thickness > 0. */
int nb_set_detector(nb_sim *sim, int n_panels, const nb_panel *panels,
                    int oversample, int n_layers, double thickness_m,
                    double atten_m);

/* Number of pixels of the detector (0 before nb_set_detector). */
long long nb_num_pixels(const nb_sim *sim);

/* Queue the Bragg-spot sum of every pixel and add it to the image (the
 * fused addArray: image[p] += (double) I_p).  Asynchronous on the handle's
 * stream.  The kernels stage the phi x mosaic and source tables in 200 KB
 * of shared memory: (18 n_phi n_mosaic + 12 n_src) x 4 bytes for NB_MIXED
 * and NB_F32, which always fits within the limits of nb_set_crystal and
 * nb_set_beam, and (9 n_phi n_mosaic + 11 n_src) x 8 bytes for NB_F64
 * (with 1024 sources, at most 1592 orientations).  Errors: NB_ESTATE
 * before crystal, beam and detector are set; NB_EINVAL if the tables
 * exceed that limit; NB_ECUDA if the launch fails. */
int nb_add_spots(nb_sim *sim);

/* As nb_add_spots for the listed global pixel indices only (a host array
 * of n_pix int64 values, copied; duplicates are added twice).  Errors:
 * NB_EINVAL for an index outside [0, nb_num_pixels). */
int nb_add_spots_pixels(nb_sim *sim, const long long *pixels, long long n_pix);

/* Set every pixel of the image to 0 (asynchronous). */
int nb_zero_image(nb_sim *sim);

/* Copy the image (n_elems must equal nb_num_pixels) to dst, converted to
 * dtype (NB_DTYPE_F32 / NB_DTYPE_F64); dst is device memory of the
 * handle's device if on_device, else host memory.  Blocks until the
 * handle's queued work and the copy are done.  Errors: NB_EINVAL for a
 * mis-sized n_elems, NULL dst or a bad dtype. */
int nb_get_image(nb_sim *sim, void *dst, size_t n_elems, int dtype,
                 int on_device);

/* Device pointer of the resident double image (for zero-copy readers on
 * the same stream); NULL before nb_set_detector. */
const double *nb_image_device_ptr(const nb_sim *sim);

/* Work counts of the last nb_add_spots* call: *pixel_steps = pixels x
 * subpixels x layers x sources x phi steps x mosaic domains; and
 * *evaluated_terms = the steps whose term was evaluated (NB_MIXED and
 * NB_F32 skip Gaussian terms whose F_latt^2 / (Na Nb Nc)^2 = exp(-2 sum
 * N^2 f^2 / 0.63) lies below exp(-88) < FLT_MIN, i.e. terms that vanish in
 * FP32; NB_F64 evaluates every step and reports 0 here).  Blocks until the
 * launch is done.  Errors: NB_EINVAL for NULL outputs. */
int nb_get_stats(nb_sim *sim, long long *evaluated_terms,
                 long long *pixel_steps);

/* Replace the values of the resident structure-factor table (Sec. II: one
 * structure factor per Bragg spot) from device memory: F holds n_elems
 * floats on the handle's device in the layout of nb_set_crystal, and
 * n_elems must equal hkl_n[0] hkl_n[1] hkl_n[2] of the table set there
 * (shape, origin, lookup and default_F are kept).  The copy is queued on
 * the handle's stream (nothing goes through the host), so the caller must
 * not change F until that stream has passed it; the tables derived
 * from F (see nb_set_crystal) are rebuilt at the next launch.  This is the refinement
 * loop's upload: a structure-factor table that already lives on the GPU
 * (a torch tensor being refined) stays there.  Errors: NB_ESTATE before
 * nb_set_crystal has set a table; NB_EINVAL for NULL F or a wrong
 * n_elems; NB_ECUDA if the copy cannot be queued. */
int nb_set_fcell_device(nb_sim *sim, const float *F, size_t n_elems);

/* Work counts of the last nb_add_spots* call, for the roofline of the work
 * the kernels perform (the Bragg-spot sum of Sec. III-B: its steps, and
 * what the warp-per-pixel kernel does to avoid visiting most of them).
 * counts[i] for i < n_counts receives (entries past NB_WORK_N are 0):
 *   NB_WORK_PIXEL_STEPS  pixels x subpixels x layers x sources x phi x mosaic
 *   NB_WORK_UNITS        pixels x subpixels x layers
 *   NB_WORK_ITEMS        units x phi steps x mosaic domains
 *   NB_WORK_INTERVALS    lattice points for which the warp kernel solved the
 *                        source interval of an item (0 for other kernels)
 *   NB_WORK_BLOCKS       (item, 8-source block) range tests of the warp
 *                        kernel's pruned scan (0 for other kernels)
 *   NB_WORK_PAIRS        steps whose fractional offset was formed and tested
 *                        against the Gaussian cut (every step for the
 *                        thread-per-pixel and FP64 kernels)
 *   NB_WORK_TERMS        steps whose term was evaluated (as nb_get_stats;
 *                        every step for NB_F64)
 * The warp kernel counts pairs, intervals and blocks only in launches made
 * with the option NB_OPT_COUNT_WORK set (a separate instantiation, so that
 * the counting costs the other launches nothing); otherwise those three
 * are -1 after a warp-kernel launch.  The counts depend only on the inputs.
 * Blocks until the launch is done.  Errors: NB_EINVAL for NULL counts or
 * n_counts < 1. */
enum { NB_WORK_PIXEL_STEPS = 0, NB_WORK_UNITS = 1, NB_WORK_ITEMS = 2,
       NB_WORK_INTERVALS = 3, NB_WORK_BLOCKS = 4, NB_WORK_PAIRS = 5,
       NB_WORK_TERMS = 6, NB_WORK_N = 7 };
int nb_get_work(nb_sim *sim, long long *counts, int n_counts);

/* Differentiable crystal (the refinement loop of x-ray tracing, Sec. II:
 * crystal parameters are refined until the simulated image matches the
 * measured one).  Sets the lab axes to the rows of Rx(tx) Ry(ty) Rz(tz) U
 * diag(a, b, c) -- axis v is cell[v] times column v of R U -- with U a
 * row-major 3x3 rotation, cell = (a, b, c) in Angstrom, rot = (tx, ty, tz)
 * in radians; and sets Na, Nb, Nc and the scale.  Keeps the mosaic, phi,
 * shape and table of the last nb_set_crystal, which must come first.
 * Errors: NB_ESTATE before nb_set_crystal; NB_EINVAL for non-positive cell
 * or N (integral N for sinc), non-finite values. */
int nb_set_crystal_params(nb_sim *sim, const double U[9], const double cell[3],
                          const double rot[3], const double ncells[3],
                          double scale);

/* Adjoint of the Bragg-spot sum.  Given dLdI (device, nb_num_pixels
 * doubles: dL/dI_p of any scalar loss L of the image), writes
 * grad = dL/d(tx, ty, tz, a, b, c, Na, Nb, Nc, scale) (host, 10 doubles)
 * and, when gradF (device, hkl_n[0] hkl_n[1] hkl_n[2] doubles) is not NULL,
 * adds dL/dF of every structure factor into it (scatter-add).  Every step
 * of the forward sum is recomputed in the FP32-mixed arithmetic; nothing
 * is stored between the passes.  With tricubic lookup F_cell's dependence
 * on hkl enters the crystal gradients and dL/dF is spread over the 64
 * stencil entries.  Blocks until done.  Needs a handle made with NB_MIXED,
 * a Gaussian shape, one source direction and nb_set_crystal_params.
 * Errors: NB_ESTATE / NB_EINVAL otherwise. */
int nb_adjoint(nb_sim *sim, const double *dLdI, double grad[10],
               double *gradF);

/* Poisson image loss L = sum_p (I_p + bkg - y_p log(I_p + bkg)) of the
 * current image against y (device, nb_num_pixels doubles); writes dL/dI_p
 * into dLdI (device, nb_num_pixels doubles) and L into *loss (host).
 * Blocks until done.  Errors: NB_EINVAL for NULL pointers or bkg <= 0. */
int nb_poisson_loss(nb_sim *sim, const double *y, double bkg, double *dLdI,
                    double *loss);

/* ------------------------------------------------------------------ */
/* Amorphous background: diffuse scatter from the air and water around the
 * crystal (the addBackground kernel of Sec. IV; the paper does not write
 * out its physics, so the convention is this library's):
 *
 *   I_p += r_e^2 fluence n_mol / os^2
 *          * sum_{sub, layer, k} F_bg(stol_k)^2 w_k cap pol omega,
 *   stol_k = |d - i_k| / (2 lambda_k)   (sin(theta)/lambda, 1/Angstrom),
 *
 * with cap, pol, omega, the subpixels, layers and sources those of the
 * spot sum, and F_bg the scattering factor of one molecule, interpolated
 * linearly between the knots of a table and held at its end values.
 *
 * nb_set_background copies the table: stol (host, n_knots strictly
 * increasing values), F (host, n_knots values) and n_molecules >= 0, the
 * number of scattering molecules in the beam.  Errors: NB_EINVAL for NULL,
 * n_knots outside [2, 4096], knots not increasing, non-finite values.
 *
 * nb_add_background queues one launch that adds the background of every
 * pixel into the handle's image (after, before or without the spots; the
 * crystal is not needed).  NB_F64 handles evaluate it in FP64.  NB_MIXED
 * and NB_F32 handles take the pixel's corner in FP64 and the rest in FP32:
 * each block of up to 32 sources is summed in four plain FP32 chains and
 * the blocks are added with compensation (within about 12 ulp of the
 * exact sum for any number of sources).  Errors: NB_ESTATE before
 * nb_set_beam, nb_set_detector and nb_set_background; NB_EINVAL if the
 * knot and source tables exceed the kernel's 200 KB of shared memory. */
int nb_set_background(nb_sim *sim, const double *stol, const double *F,
                      int n_knots, double n_molecules);
int nb_add_background(nb_sim *sim);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of shot requests on one GPU.  The paper
 * hides I/O latency by sharing a GPU between several ranks, each with its
 * own batch of images (Sec. IV, Fig. 3); here one server keeps the
 * structure-factor table and the detector resident and admits requests of
 * uneven size as slots and image memory free up, batching all running
 * requests into each launch. */
typedef struct nb_server nb_server; /* opaque, owned by the library */

enum { NB_REQ_UNKNOWN = -1, NB_REQ_QUEUED = 0, NB_REQ_RUNNING = 1,
       NB_REQ_DONE = 2 };

/* Create a server on `device`, queuing work on `cuda_stream` (a
 * non-default cudaStream_t, or NULL: the server makes its own).
 *   max_slots    requests resident at once (1..4096; each slot holds up to
 *                64 mosaic domains and 128 sources).
 *   pool_bytes   device memory for the images of resident requests (FP64,
 *                8 bytes per ROI pixel); admission needs room here.
 *   step_budget  pixel-steps per scheduling step (<= 0: 1e9).
 *   panel ...    the resident detector (one panel), oversample, layers.
 *   F ...        the resident structure-factor table (copied).
 *   Na, Nb, Nc   Gaussian lattice shape (the only shape served).
 *   dir, fluence, kahn_K, e_vec   beam direction shared by all sources,
 *                fluence, polarization.
 * Every step is one replay of one of two CUDA graphs, used in turn: the
 * work-list upload from that graph's pinned buffer, a counter reset and
 * two persistent kernels whose blocks pull work items, 128 pixels for the
 * thread-per-pixel kernel and 64 pixels for the warp-per-pixel kernel
 * (which takes requests with tricubic lookup and >= 8 mosaic domains).
 * Errors: NB_EINVAL (bad sizes), NB_ENOMEM, NB_ECUDA. */
int nb_server_create(nb_server **out, int device, void *cuda_stream,
                     int max_slots, long long pool_bytes,
                     long long step_budget, const nb_panel *panel,
                     int oversample, int n_layers, double thickness_m,
                     double atten_m, const float *F, const int hkl_min[3],
                     const int hkl_n[3], int interp, double default_F,
                     double Na, double Nb, double Nc, const double dir[3],
                     double fluence, double kahn_K, const double e_vec[3]);

/* Queue one shot: lab axes (rows a, b, c), n_mosaic domain matrices,
 * n_src wavelengths and weights, scale, and the ROI (a rectangle of the
 * resident panel).  Inputs are copied.  *request_id receives its id.
 * Errors: NB_EINVAL for sizes beyond a slot, an ROI outside the panel or
 * larger than the whole pool. */
int nb_server_submit(nb_server *srv, const double axes[9],
                     const double *umats, int n_mosaic,
                     const double *lambda_A, const double *weights,
                     int n_src, double scale, int roi_f0, int roi_s0,
                     int roi_nf, int roi_ns, long long *request_id);

/* One scheduling step: admit queued requests (FIFO; a request that does
 * not fit may be passed by later ones until it has waited 8 steps), cut
 * the running requests into work items up to the pixel-step budget (half
 * of it shared equally by the running requests, at least one item each;
 * the rest to the oldest requests first) and
 * queue them on the GPU, then wait (up to timeout_s seconds)
 * for the step queued by the previous call, so that one step runs while
 * the next is prepared.  When there is nothing new to queue, the call
 * waits for every step in flight.  A request completes when the step
 * holding its last work item has finished: its slot is released and its
 * image stays in the pool until fetched.  *n_active (may be NULL) =
 * queued + running.  Errors: NB_ETIMEOUT if a step waited for is still
 * running after timeout_s (a later call waits for it again); NB_ESTATE if
 * requests are queued but nothing runs, none can be admitted and the call
 * completed nothing (the pool is held by unfetched results: fetch them);
 * NB_ECUDA. */
int nb_server_step(nb_server *srv, double timeout_s, int *n_active);

/* Ids of requests completed since the last call (up to max_ids); a
 * request fetched with nb_server_result before it was reported is not
 * reported. */
int nb_server_completed(nb_server *srv, long long *ids, int max_ids,
                        int *n_out);

/* State of a request: NB_REQ_QUEUED, NB_REQ_RUNNING, NB_REQ_DONE, or
 * NB_REQ_UNKNOWN (never submitted, or already fetched). */
int nb_server_state(nb_server *srv, long long request_id, int *state);

/* Copy a completed request's image (ROI pixels, slow-major, FP64:
 * dtype must be NB_DTYPE_F64) to dst (device memory if on_device, else
 * host), then release its pool memory.  A server only admits new requests
 * while pool memory is free, so fetch results.
 * Errors: NB_ESTATE if not done; NB_EINVAL for a wrong size or id. */
int nb_server_result(nb_server *srv, long long request_id, void *dst,
                     size_t n_elems, int dtype, int on_device);

/* Queue lengths and free pool bytes (any pointer may be NULL). */
int nb_server_info(const nb_server *srv, long long *queued,
                   long long *running, long long *done,
                   long long *pool_free_bytes);

/* Text of the server's last error. */
const char *nb_server_last_error(const nb_server *srv);

/* Free the server (waits for its work); NULL is a no-op. */
int nb_server_free(nb_server *srv);

/* Tuning options (nb_set_option keys). */
enum {
    /* kernel variant of NB_MIXED: NB_VARIANT_AUTO (default: one warp per
     * pixel for Gaussian shapes with tricubic lookup, <= 32 subpixel x layer
     * units and >= 8 (unit, phi x mosaic) items per pixel, else one thread
     * per pixel), NB_VARIANT_THREAD, NB_VARIANT_WARP (Gaussian shapes with
     * <= 32 units only; falls back to NB_VARIANT_THREAD otherwise) */
    NB_OPT_VARIANT = 1,
    /* 1: launches of the warp-per-pixel kernel also count the work
     * nb_get_work reports (pairs, intervals, block tests); 0 (default):
     * they do not, and run the instantiation without the counters */
    NB_OPT_COUNT_WORK = 2,
    /* a test hook for the failure paths, not part of the method: the next
     * `value` device allocations made for simulation handles (any nb_sim
     * of the process; the server and the FP64 peak probe allocate on their
     * own) fail as if the device were out of memory (0, the default, turns
     * it off).  A call whose own buffer is refused returns
     * NB_ENOMEM and leaves the handle usable (the same call succeeds once
     * memory is there); a launch whose table derived from F is refused
     * (nb_set_crystal lists them) reads F itself and gives the same
     * result. */
    NB_OPT_FAIL_ALLOCS = 3
};
enum { NB_VARIANT_AUTO = 0, NB_VARIANT_THREAD = 1, NB_VARIANT_WARP = 2 };

/* Set a tuning option; results agree across variants within the precision's
 * tolerance.  Errors: NB_EINVAL for an unknown key or value. */
int nb_set_option(nb_sim *sim, int key, long long value);

/* Bragg-spot sum without any allocation by the library.  The paper has no
 * counterpart: this exists for callers that must not call cudaMalloc (for
 * example code whose device memory all comes from its own pool or arena,
 * or a plug-in whose host forbids device allocations).  It runs the
 * NB_MIXED one-warp-per-pixel kernel for a Gaussian shape on one panel and
 * adds the result to `image`.
 *
 * Device pointers (caller-owned, on the calling thread's current device):
 *   axes_pm    n_pm x 9 doubles, rows a, b, c (Angstrom) of each crystal
 *              orientation U_m R_phi (a, b, c)_lab, already rotated by the
 *              caller; the sum averages over the n_pm entries.
 *   F          structure factors as for nb_set_crystal.
 *   lambda_A, weights   n_src doubles each.
 *   image      nfast x nslow doubles (slow-major), accumulated into.
 * Host values: panel (copied), oversample and n_layers (os^2 x layers <=
 * 32), thickness_m, atten_m, Na, Nb, Nc, scale, hkl_min, hkl_n, interp,
 * default_F, dir (the one propagation direction of every source), fluence,
 * kahn_K, e_vec, as for the other calls; cuda_stream a cudaStream_t.
 *
 * Scratch: a file-scope device array of about 200 KB on every GPU that
 * loads the library (held until the process exits) holds the staged tables
 * and two counters; n_pm <= 2048 and n_src <= 1024 are the limits it fits,
 * and larger values return NB_EINVAL.  The kernel also stages those
 * tables, with its per-warp rings, in at most 200 KB (204800 bytes) of
 * shared memory: (72 n_pm + 48 n_src + 5120, rounded up to a multiple of
 * 16) + 8 ceil(n_src / 8) + 4 n_src + 28800 bytes must fit, so the two limits
 * cannot both be reached: with n_pm = 2048 at most 441 sources are
 * accepted, with n_src = 1024 at most 1619 orientations.  A pair beyond
 * that returns NB_EINVAL before anything is queued.  Every call shares the
 * array and
 * rewrites it (the counters are cleared before the kernel runs), so calls
 * whose work overlaps on the GPU race: serialise them.  The first call on a
 * device looks up the array's device address once (cudaGetSymbolAddress
 * with that device current): make that first call before any stream
 * capture.  Each call waits on the host for its table set-up on
 * `cuda_stream` (an 8-byte device-to-host read), then queues the kernel
 * asynchronously.
 * Errors: NB_EINVAL for NULL pointers, sizes outside the limits above, a
 * non-unit dir, e_vec parallel to dir, or bad geometry; NB_ECUDA if a CUDA
 * call fails. */
int nb_add_spots_noalloc(const nb_panel *panel, int oversample, int n_layers,
                         double thickness_m, double atten_m,
                         const double *axes_pm, int n_pm, double Na,
                         double Nb, double Nc, double scale, const float *F,
                         const int hkl_min[3], const int hkl_n[3], int interp,
                         double default_F, const double *lambda_A,
                         const double *weights, int n_src,
                         const double dir[3], double fluence, double kahn_K,
                         const double e_vec[3], double *image,
                         void *cuda_stream);

/* Wait for the handle's queued work. */
int nb_synchronize(nb_sim *sim);

/* Measured FP64 FMA throughput of `device`, in TFLOP/s (an FMA counts as
 * two flops), written to *tflops.  Not part of the method: the ceiling
 * against which the NB_F64 kernels, which issue scalar FP64 FMAs, are
 * measured.  A kernel of independent FMA chains in 4 blocks of 256
 * threads per SM runs once to warm up and three times timed with CUDA
 * events on a private stream; the best time counts (about 10 ms per launch
 * on a GB300).  Blocks the caller until done and restores the calling
 * thread's current device.  Errors: NB_EINVAL for a NULL tflops or a
 * device outside [0, device count); NB_ENOMEM if its small result buffer
 * cannot be allocated; NB_ECUDA if a CUDA call fails (*tflops is then 0). */
int nb_fp64_peak_tflops(int device, double *tflops);

/* Free the handle and everything it owns; NULL is a no-op. */
int nb_free(nb_sim *sim);

/* Text of the last error on this handle ("" if none; a static string for a
 * NULL handle).  Valid until the next call on the handle. */
const char *nb_last_error(const nb_sim *sim);

/* Library version string. */
const char *nb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NBGB_H */
