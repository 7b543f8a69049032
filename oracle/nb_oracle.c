/*
 * nb_oracle.c -- plain FP64 CPU oracle for the per-pixel Bragg-spot sum
 * (the nanoBraggSpots kernel of Sec. III-B: every detector pixel is
 * simulated independently; the sum runs over crystal orientation,
 * mosaicity and photon energy; each Bragg spot carries one structure
 * factor, Sec. II).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  The product path (the
 * CUDA library) never does, and the two share no code: not a header, not a
 * helper, not a table.  Inputs reach both sides from the seeded generators,
 * nothing else is shared.
 *
 * The paper prints no formula for this sum, so the oracle writes out the
 * textbook kinematic-diffraction definition in the order of the loops:
 *
 *   for pixel p, subpixel (i, j), thickness layer t:
 *     P  = O + (f + (i+1/2)/os) px fdir + (s + (j+1/2)/os) px sdir + t dt n
 *     R  = |P|, d = P / R
 *     omega = px^2 (n . P) / R^3                 solid angle, full pixel area
 *     cap   = exp(-t dt/(l rho)) - exp(-(t+1) dt/(l rho)),  rho = d . n
 *             (1 when the sensor has no thickness)
 *     for source k:      S = (d - i_k) / lambda_k,  pol = Kahn(d, i_k, K, e)
 *       for phi step j, mosaic domain m:
 *         (a, b, c) = U_m R_phi(j) (a, b, c)_lab
 *         h = a.S, k = b.S, l = c.S
 *         acc += F_cell(hkl)^2 F_latt(hkl)^2 w_k cap pol omega
 *   I_p = r_e^2 fluence scale acc / (os^2 M Phi)
 *
 * with
 *   sinc  F_latt = prod_axes sin(pi N h) / sin(pi h)      (-> N at integer h)
 *   gauss F_latt = Na Nb Nc exp(-(Na^2 fh^2 + Nb^2 fk^2 + Nc^2 fl^2) / 0.63),
 *         f = h - h0, h0 = ceil(h - 1/2) (ties round down)
 *   nearest  F_cell = F[h0, k0, l0], default_F outside the table
 *   tricubic F_cell = 4-point Lagrange interpolation of F along each axis on
 *            nodes floor(h)-1 .. floor(h)+2; nearest if that stencil leaves
 *            the table.
 *   Kahn  pol = (1 + cos^2 2theta - K cos 2psi sin^2 2theta) / 2, cos 2theta =
 *         d . i, psi the azimuth of d about i measured from the E vector.
 *
 * Every point the paper leaves open is fixed by one of the readings above.
 *
 * The differentiable form (orc_loss_grad) parametrises the lab-frame axes as
 * rows of Rx(tx) Ry(ty) Rz(tz) U diag(a, b, c): an orthorhombic cell with
 * lengths a, b, c, a fixed orientation U and three small rotation angles,
 * and returns the Poisson loss L = sum_p (I_p + bkg - y_p log(I_p + bkg))
 * with its gradient w.r.t. (tx, ty, tz, a, b, c, Na, Nb, Nc, scale) and
 * every structure factor (Gaussian shape; nearest or tricubic lookup, the
 * latter through the derivative of the Lagrange weights).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
/* classical electron radius in metres (CODATA 2018) */
#define ORC_RE 2.8179403262e-15

typedef struct {
    /* crystal */
    double axes[9];          /* rows a, b, c in Angstrom, lab frame       */
    const double *umats;     /* n_mosaic x 9, row-major                    */
    int n_mosaic;
    int n_phi;
    double phi0_deg;
    double phistep_deg;
    double spindle[3];
    double ncells[3];
    int shape;               /* 0 sinc, 1 gauss                            */
    double scale;
    const double *F;         /* hkl_n[0] x hkl_n[1] x hkl_n[2], l fastest  */
    int hkl_min[3];
    int hkl_n[3];
    int interp;              /* 0 nearest, 1 tricubic                      */
    double default_F;
    /* beam */
    const double *dirs;      /* n_src x 3 unit propagation directions      */
    const double *lambdas;   /* Angstrom                                   */
    const double *weights;
    int n_src;
    double fluence;          /* photons per m^2                            */
    double kahn;
    double evec[3];
    /* detector */
    int n_panels;
    const double *panel_geom; /* 13 per panel: origin, fdir, sdir, ndir, px */
    const int *panel_dims;    /* 2 per panel: nfast, nslow                  */
    int oversample;
    int n_layers;
    double thickness;        /* m */
    double atten;            /* m */
    int sinc_mode;           /* 0 literal sin(pi N h)/sin(pi h), 1 reduced  */
} orc_params;

/* ---------------------------------------------------------------- basics */

static double dot3(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static void matvec3(const double *M, const double *v, double *o)
{
    for (int r = 0; r < 3; ++r)
        o[r] = M[3 * r] * v[0] + M[3 * r + 1] * v[1] + M[3 * r + 2] * v[2];
}

/* rotation of v about the unit axis k by ang radians (Rodrigues) */
static void rotate_about(const double *v, const double *k, double ang,
                         double *o)
{
    double c = cos(ang), s = sin(ang), kv = dot3(k, v), kxv[3];
    cross3(k, v, kxv);
    for (int i = 0; i < 3; ++i)
        o[i] = v[i] * c + kxv[i] * s + k[i] * kv * (1.0 - c);
}

/* nearest integer, ties rounded down */
static double nearest_int(double x) { return ceil(x - 0.5); }

/* ------------------------------------------------------- lattice factor */

double orc_sincg(double h, double N, int mode)
{
    int integral = (N == floor(N));
    if (mode == 0 || !integral) {
        double den = sin(ORC_PI * h);
        if (den == 0.0)
            return N;
        return sin(ORC_PI * N * h) / den;
    }
    /* sin(pi N (n + f)) / sin(pi (n + f)) = (-1)^(n (N - 1)) sin(pi N f) /
     * sin(pi f) for integer n and N */
    double n = nearest_int(h);
    double f = h - n;
    double sgn = (fmod(fabs(n) * (N - 1.0), 2.0) == 0.0) ? 1.0 : -1.0;
    if (f == 0.0)
        return sgn * N;
    return sgn * sin(ORC_PI * N * f) / sin(ORC_PI * f);
}

double orc_flatt(const orc_params *p, const double *hkl)
{
    if (p->shape == 0) {
        return orc_sincg(hkl[0], p->ncells[0], p->sinc_mode) *
               orc_sincg(hkl[1], p->ncells[1], p->sinc_mode) *
               orc_sincg(hkl[2], p->ncells[2], p->sinc_mode);
    }
    double rad2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double f = hkl[a] - nearest_int(hkl[a]);
        rad2 += p->ncells[a] * p->ncells[a] * f * f;
    }
    return p->ncells[0] * p->ncells[1] * p->ncells[2] * exp(-rad2 / 0.63);
}

/* ------------------------------------------------------ structure factor */

static int in_table(const orc_params *p, long ih, long ik, long il)
{
    return ih >= p->hkl_min[0] && ih < p->hkl_min[0] + p->hkl_n[0] &&
           ik >= p->hkl_min[1] && ik < p->hkl_min[1] + p->hkl_n[1] &&
           il >= p->hkl_min[2] && il < p->hkl_min[2] + p->hkl_n[2];
}

static double table_entry(const orc_params *p, long ih, long ik, long il)
{
    long i = ih - p->hkl_min[0], j = ik - p->hkl_min[1],
         k = il - p->hkl_min[2];
    return p->F[(i * p->hkl_n[1] + j) * p->hkl_n[2] + k];
}

/* 4-point Lagrange weights for nodes -1, 0, 1, 2 at x */
static void lagrange4(double x, double *w)
{
    w[0] = -x * (x - 1.0) * (x - 2.0) / 6.0;
    w[1] = (x + 1.0) * (x - 1.0) * (x - 2.0) / 2.0;
    w[2] = -(x + 1.0) * x * (x - 2.0) / 2.0;
    w[3] = (x + 1.0) * x * (x - 1.0) / 6.0;
}

/* derivatives of the 4-point Lagrange weights at x */
static void lagrange4_deriv(double x, double *w)
{
    w[0] = -(3.0 * x * x - 6.0 * x + 2.0) / 6.0;
    w[1] = (3.0 * x * x - 4.0 * x - 1.0) / 2.0;
    w[2] = -(3.0 * x * x - 2.0 * x - 2.0) / 2.0;
    w[3] = (3.0 * x * x - 1.0) / 6.0;
}

static size_t table_index(const orc_params *p, long ih, long ik, long il)
{
    return ((size_t)(ih - p->hkl_min[0]) * p->hkl_n[1] +
            (size_t)(ik - p->hkl_min[1])) * p->hkl_n[2] +
           (size_t)(il - p->hkl_min[2]);
}

/* F_cell at hkl with its gradient dF[3] = dF_cell/dh, and the table
 * entries F_cell is a linear combination of: idx[n], coef[n] (n <= 64; n = 0
 * for default_F).  Returns n. */
int orc_fcell_lin(const orc_params *p, const double *hkl, double *Fc,
                  double *dF, size_t *idx, double *coef)
{
    dF[0] = dF[1] = dF[2] = 0.0;
    if (p->interp == 1) {
        long fl[3];
        for (int a = 0; a < 3; ++a)
            fl[a] = (long)floor(hkl[a]);
        if (in_table(p, fl[0] - 1, fl[1] - 1, fl[2] - 1) &&
            in_table(p, fl[0] + 2, fl[1] + 2, fl[2] + 2)) {
            double w[3][4], d[3][4];
            for (int a = 0; a < 3; ++a) {
                lagrange4(hkl[a] - fl[a], w[a]);
                lagrange4_deriv(hkl[a] - fl[a], d[a]);
            }
            int n = 0;
            double v = 0.0;
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j)
                    for (int k = 0; k < 4; ++k) {
                        size_t e = table_index(p, fl[0] - 1 + i,
                                               fl[1] - 1 + j, fl[2] - 1 + k);
                        double F = p->F[e];
                        double c = w[0][i] * w[1][j] * w[2][k];
                        v += c * F;
                        dF[0] += d[0][i] * w[1][j] * w[2][k] * F;
                        dF[1] += w[0][i] * d[1][j] * w[2][k] * F;
                        dF[2] += w[0][i] * w[1][j] * d[2][k] * F;
                        idx[n] = e;
                        coef[n] = c;
                        ++n;
                    }
            *Fc = v;
            return n;
        }
    }
    long h0 = (long)nearest_int(hkl[0]), k0 = (long)nearest_int(hkl[1]),
         l0 = (long)nearest_int(hkl[2]);
    if (in_table(p, h0, k0, l0)) {
        idx[0] = table_index(p, h0, k0, l0);
        coef[0] = 1.0;
        *Fc = p->F[idx[0]];
        return 1;
    }
    *Fc = p->default_F;
    return 0;
}

double orc_fcell(const orc_params *p, const double *hkl)
{
    if (p->interp == 1) {
        long fl[3];
        for (int a = 0; a < 3; ++a)
            fl[a] = (long)floor(hkl[a]);
        if (in_table(p, fl[0] - 1, fl[1] - 1, fl[2] - 1) &&
            in_table(p, fl[0] + 2, fl[1] + 2, fl[2] + 2)) {
            double wh[4], wk[4], wl[4], sum = 0.0;
            lagrange4(hkl[0] - fl[0], wh);
            lagrange4(hkl[1] - fl[1], wk);
            lagrange4(hkl[2] - fl[2], wl);
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j)
                    for (int k = 0; k < 4; ++k)
                        sum += wh[i] * wk[j] * wl[k] *
                               table_entry(p, fl[0] - 1 + i, fl[1] - 1 + j,
                                           fl[2] - 1 + k);
            return sum;
        }
    }
    long h0 = (long)nearest_int(hkl[0]), k0 = (long)nearest_int(hkl[1]),
         l0 = (long)nearest_int(hkl[2]);
    if (in_table(p, h0, k0, l0))
        return table_entry(p, h0, k0, l0);
    return p->default_F;
}

/* ---------------------------------------------------- per-pixel factors */

double orc_polar(const double *d, const double *inc, double K,
                 const double *e)
{
    double c2t = dot3(d, inc);
    double c2 = c2t * c2t;
    if (K == 0.0)
        return 0.5 * (1.0 + c2);
    double ep[3], bp[3], ei = dot3(e, inc), nrm;
    for (int i = 0; i < 3; ++i)
        ep[i] = e[i] - ei * inc[i];
    nrm = sqrt(dot3(ep, ep));
    for (int i = 0; i < 3; ++i)
        ep[i] /= nrm;
    cross3(inc, ep, bp);
    double psi = atan2(dot3(d, bp), dot3(d, ep));
    return 0.5 * (1.0 + c2 - K * cos(2.0 * psi) * (1.0 - c2));
}

double orc_omega(double px, const double *n, const double *P)
{
    double R = sqrt(dot3(P, P));
    return px * px * dot3(n, P) / (R * R * R);
}

double orc_capture(int t, double dt, double atten, double rho,
                   double thickness)
{
    if (thickness == 0.0)
        return 1.0;
    return exp(-t * dt / (atten * rho)) - exp(-(t + 1) * dt / (atten * rho));
}

/* ------------------------------------------------------------- the sum */

/* rows a, b, c of U_m R_phi(j) applied to the lab axes, for every (j, m) */
static void rotated_axes(const orc_params *p, double *ax)
{
    double k[3], nk = sqrt(dot3(p->spindle, p->spindle));
    for (int i = 0; i < 3; ++i)
        k[i] = p->spindle[i] / nk;
    for (int j = 0; j < p->n_phi; ++j) {
        double phi = (p->phi0_deg + j * p->phistep_deg) * ORC_PI / 180.0;
        for (int m = 0; m < p->n_mosaic; ++m) {
            for (int v = 0; v < 3; ++v) {
                double r[3];
                rotate_about(p->axes + 3 * v, k, phi, r);
                matvec3(p->umats + 9 * m, r,
                        ax + ((size_t)j * p->n_mosaic + m) * 9 + 3 * v);
            }
        }
    }
}

static void locate(const orc_params *p, long long g, int *panel, long *s,
                   long *f)
{
    for (int q = 0; q < p->n_panels; ++q) {
        long long np = (long long)p->panel_dims[2 * q] * p->panel_dims[2 * q + 1];
        if (g < np) {
            *panel = q;
            *s = (long)(g / p->panel_dims[2 * q]);
            *f = (long)(g % p->panel_dims[2 * q]);
            return;
        }
        g -= np;
    }
    *panel = -1;
}

static double pixel_value(const orc_params *p, const double *ax, int q,
                          long s, long f)
{
    const double *G = p->panel_geom + 13 * q;
    const double *O = G, *fd = G + 3, *sd = G + 6, *nd = G + 9;
    double px = G[12];
    int os = p->oversample;
    double dt = p->n_layers > 0 ? p->thickness / p->n_layers : 0.0;
    double acc = 0.0;
    for (int i = 0; i < os; ++i) {
        for (int j = 0; j < os; ++j) {
            for (int t = 0; t < p->n_layers; ++t) {
                double P[3], d[3];
                for (int c = 0; c < 3; ++c)
                    P[c] = O[c] + (f + (i + 0.5) / os) * px * fd[c] +
                           (s + (j + 0.5) / os) * px * sd[c] +
                           t * dt * nd[c];
                double R = sqrt(dot3(P, P));
                for (int c = 0; c < 3; ++c)
                    d[c] = P[c] / R;
                double omega = orc_omega(px, nd, P);
                double rho = dot3(d, nd);
                double cap = orc_capture(t, dt, p->atten, rho, p->thickness);
                for (int k = 0; k < p->n_src; ++k) {
                    const double *inc = p->dirs + 3 * k;
                    double S[3];
                    for (int c = 0; c < 3; ++c)
                        S[c] = (d[c] - inc[c]) / p->lambdas[k];
                    double pol = orc_polar(d, inc, p->kahn, p->evec);
                    for (int jm = 0; jm < p->n_phi * p->n_mosaic; ++jm) {
                        const double *A = ax + (size_t)jm * 9;
                        double hkl[3] = {dot3(A, S), dot3(A + 3, S),
                                         dot3(A + 6, S)};
                        double Fl = orc_flatt(p, hkl);
                        double Fc = orc_fcell(p, hkl);
                        acc += Fc * Fc * Fl * Fl * p->weights[k] * cap * pol *
                               omega;
                    }
                }
            }
        }
    }
    return ORC_RE * ORC_RE * p->fluence * p->scale * acc /
           ((double)os * os * p->n_mosaic * p->n_phi);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* image values of the pixels pix[0..n) (global index: panel-major, then
 * slow, then fast); returns 0, or -1 on a bad pixel index */
int orc_image(const orc_params *p, const long long *pix, long long n,
              double *out, int nthreads)
{
    size_t nax = (size_t)p->n_phi * p->n_mosaic * 9;
    double *ax = (double *)malloc(nax * sizeof(double));
    if (!ax)
        return -2;
    rotated_axes(p, ax);
    int bad = 0;
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads) reduction(| : bad)
#endif
    for (long long i = 0; i < n; ++i) {
        int q;
        long s, f;
        locate(p, pix[i], &q, &s, &f);
        if (q < 0) {
            bad = 1;
            out[i] = 0.0;
            continue;
        }
        out[i] = pixel_value(p, ax, q, s, f);
    }
    free(ax);
    return bad ? -1 : 0;
}

/* ------------------------------------------------ amorphous background */
/*
 * Diffuse scatter from the air and water around the crystal (the
 * addBackground kernel of Sec. IV).  The paper names the kernel but not its
 * physics; the convention here is ours:
 *
 *   for pixel p, subpixel (i, j), thickness layer t   (P, d, omega, cap as
 *   in the spot sum), source k:
 *     stol  = |d - i_k| / (2 lambda_k)            sin(theta) / lambda
 *     F_bg  = the (stol, F) table interpolated linearly between its knots,
 *             held at the end values outside them
 *     acc  += F_bg^2 w_k cap pol omega
 *   I_p = r_e^2 fluence n_mol acc / os^2
 *
 * n_mol is the number of scattering molecules in the beam; the table holds
 * the scattering factor of one molecule.  Nothing here depends on the
 * crystal.
 */

double orc_bg_factor(const double *stol, const double *F, int n, double x)
{
    if (x <= stol[0])
        return F[0];
    if (x >= stol[n - 1])
        return F[n - 1];
    int j = 0;
    while (stol[j + 1] <= x)
        ++j;
    double t = (x - stol[j]) / (stol[j + 1] - stol[j]);
    return F[j] + t * (F[j + 1] - F[j]);
}

static double background_value(const orc_params *p, const double *stol,
                               const double *Fbg, int nk, double n_mol,
                               int q, long s, long f)
{
    const double *G = p->panel_geom + 13 * q;
    const double *O = G, *fd = G + 3, *sd = G + 6, *nd = G + 9;
    double px = G[12];
    int os = p->oversample;
    double dt = p->n_layers > 0 ? p->thickness / p->n_layers : 0.0;
    double acc = 0.0;
    for (int i = 0; i < os; ++i)
        for (int j = 0; j < os; ++j)
            for (int t = 0; t < p->n_layers; ++t) {
                double P[3], d[3];
                for (int c = 0; c < 3; ++c)
                    P[c] = O[c] + (f + (i + 0.5) / os) * px * fd[c] +
                           (s + (j + 0.5) / os) * px * sd[c] +
                           t * dt * nd[c];
                double R = sqrt(dot3(P, P));
                for (int c = 0; c < 3; ++c)
                    d[c] = P[c] / R;
                double omega = orc_omega(px, nd, P);
                double cap = orc_capture(t, dt, p->atten, dot3(d, nd),
                                         p->thickness);
                for (int k = 0; k < p->n_src; ++k) {
                    const double *inc = p->dirs + 3 * k;
                    double v[3];
                    for (int c = 0; c < 3; ++c)
                        v[c] = d[c] - inc[c];
                    double x = sqrt(dot3(v, v)) / (2.0 * p->lambdas[k]);
                    double Fb = orc_bg_factor(stol, Fbg, nk, x);
                    double pol = orc_polar(d, inc, p->kahn, p->evec);
                    acc += Fb * Fb * p->weights[k] * cap * pol * omega;
                }
            }
    return ORC_RE * ORC_RE * p->fluence * n_mol * acc / ((double)os * os);
}

/* background values of the pixels pix[0..n); returns 0, or -1 on a bad
 * pixel index or table (fewer than 2 knots, knots not increasing) */
int orc_background(const orc_params *p, const double *stol, const double *F,
                   int nk, double n_mol, const long long *pix, long long n,
                   double *out, int nthreads)
{
    if (nk < 2)
        return -1;
    for (int j = 0; j + 1 < nk; ++j)
        if (!(stol[j + 1] > stol[j]))
            return -1;
    int bad = 0;
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads) reduction(| : bad)
#endif
    for (long long i = 0; i < n; ++i) {
        int q;
        long s, f;
        locate(p, pix[i], &q, &s, &f);
        if (q < 0) {
            bad = 1;
            out[i] = 0.0;
            continue;
        }
        out[i] = background_value(p, stol, F, nk, n_mol, q, s, f);
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------ differentiable form */

static void rot_x(double t, double *M, int deriv)
{
    double c = cos(t), s = sin(t);
    double R[9] = {1, 0, 0, 0, c, -s, 0, s, c};
    double D[9] = {0, 0, 0, 0, -s, -c, 0, c, -s};
    memcpy(M, deriv ? D : R, sizeof R);
}

static void rot_y(double t, double *M, int deriv)
{
    double c = cos(t), s = sin(t);
    double R[9] = {c, 0, s, 0, 1, 0, -s, 0, c};
    double D[9] = {-s, 0, c, 0, 0, 0, -c, 0, -s};
    memcpy(M, deriv ? D : R, sizeof R);
}

static void rot_z(double t, double *M, int deriv)
{
    double c = cos(t), s = sin(t);
    double R[9] = {c, -s, 0, s, c, 0, 0, 0, 1};
    double D[9] = {-s, -c, 0, c, -s, 0, 0, 0, 0};
    memcpy(M, deriv ? D : R, sizeof R);
}

static void matmul3(const double *A, const double *B, double *C)
{
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] +
                           A[3 * i + 2] * B[6 + j];
    memcpy(C, T, sizeof T);
}

/* lab axes (rows a, b, c) of Rx(tx) Ry(ty) Rz(tz) U diag(cell) and their
 * derivatives w.r.t. tx, ty, tz, a, b, c (d_axes: 6 x 9) */
void orc_param_axes(const double *U, const double *cell, const double *rot,
                    double *axes, double *d_axes)
{
    double Rx[9], Ry[9], Rz[9], dRx[9], dRy[9], dRz[9];
    rot_x(rot[0], Rx, 0);
    rot_y(rot[1], Ry, 0);
    rot_z(rot[2], Rz, 0);
    rot_x(rot[0], dRx, 1);
    rot_y(rot[1], dRy, 1);
    rot_z(rot[2], dRz, 1);
    double M[6][9], T[9];
    /* M[0] = R U, M[1..3] = dR/dt U */
    matmul3(Ry, Rz, T);
    matmul3(Rx, T, M[0]);
    matmul3(M[0], U, M[0]);
    matmul3(Ry, Rz, T);
    matmul3(dRx, T, M[1]);
    matmul3(M[1], U, M[1]);
    matmul3(dRy, Rz, T);
    matmul3(Rx, T, M[2]);
    matmul3(M[2], U, M[2]);
    matmul3(Ry, dRz, T);
    matmul3(Rx, T, M[3]);
    matmul3(M[3], U, M[3]);
    /* axis v is column v of R U scaled by cell[v] */
    for (int v = 0; v < 3; ++v)
        for (int c = 0; c < 3; ++c)
            axes[3 * v + c] = M[0][3 * c + v] * cell[v];
    if (!d_axes)
        return;
    memset(d_axes, 0, 6 * 9 * sizeof(double));
    for (int r = 0; r < 3; ++r)
        for (int v = 0; v < 3; ++v)
            for (int c = 0; c < 3; ++c)
                d_axes[9 * r + 3 * v + c] = M[1 + r][3 * c + v] * cell[v];
    for (int v = 0; v < 3; ++v)
        for (int c = 0; c < 3; ++c)
            d_axes[9 * (3 + v) + 3 * v + c] = M[0][3 * c + v];
}

/* gradient-weighted step sum of one pixel: adds w_p * dI_p/d(param) to g
 * (10 scalars) and w_p * dI_p/dF to gF; ax/dax are the rotated axes and
 * their derivatives w.r.t. (tx, ty, tz, a, b, c) */
static void pixel_grad(const orc_params *p, const double *ax,
                       const double *dax, int q, long s, long f, double I,
                       double w_p, double *g, double *gF)
{
    const double *G = p->panel_geom + 13 * q;
    const double *O = G, *fd = G + 3, *sd = G + 6, *nd = G + 9;
    double px = G[12];
    int os = p->oversample, PM = p->n_phi * p->n_mosaic;
    double dt = p->n_layers > 0 ? p->thickness / p->n_layers : 0.0;
    /* I_p = Kc * scale * sum_steps(term) */
    double Kc = ORC_RE * ORC_RE * p->fluence /
                ((double)os * os * p->n_mosaic * p->n_phi);
    const double *N = p->ncells;
    double dacc[9] = {0};
    for (int i = 0; i < os; ++i)
        for (int j = 0; j < os; ++j)
            for (int t = 0; t < p->n_layers; ++t) {
                double P[3], d[3];
                for (int c = 0; c < 3; ++c)
                    P[c] = O[c] + (f + (i + 0.5) / os) * px * fd[c] +
                           (s + (j + 0.5) / os) * px * sd[c] + t * dt * nd[c];
                double R = sqrt(dot3(P, P));
                for (int c = 0; c < 3; ++c)
                    d[c] = P[c] / R;
                double omega = orc_omega(px, nd, P);
                double cap = orc_capture(t, dt, p->atten, dot3(d, nd),
                                         p->thickness);
                for (int k = 0; k < p->n_src; ++k) {
                    const double *inc = p->dirs + 3 * k;
                    double S[3];
                    for (int c = 0; c < 3; ++c)
                        S[c] = (d[c] - inc[c]) / p->lambdas[k];
                    double wfac = p->weights[k] * cap *
                                  orc_polar(d, inc, p->kahn, p->evec) * omega;
                    for (int jm = 0; jm < PM; ++jm) {
                        const double *A = ax + (size_t)jm * 9;
                        double hkl[3] = {dot3(A, S), dot3(A + 3, S),
                                         dot3(A + 6, S)};
                        double Fl = orc_flatt(p, hkl);
                        double Fc, dFc[3], lin_c[64];
                        size_t lin_i[64];
                        int nlin = orc_fcell_lin(p, hkl, &Fc, dFc, lin_i,
                                                 lin_c);
                        double term = Fc * Fc * Fl * Fl * wfac;
                        double fr[3], dterm[3];
                        for (int a = 0; a < 3; ++a) {
                            fr[a] = hkl[a] - nearest_int(hkl[a]);
                            /* d term / d h_a: the lattice factor through
                             * f_a, the structure factor through h_a */
                            dterm[a] = term * (-4.0 * N[a] * N[a] * fr[a] / 0.63) +
                                       2.0 * Fc * dFc[a] * Fl * Fl * wfac;
                        }
                        for (int r = 0; r < 6; ++r) {
                            const double *dA = dax + ((size_t)jm * 6 + r) * 9;
                            dacc[r] += dterm[0] * dot3(dA, S) +
                                       dterm[1] * dot3(dA + 3, S) +
                                       dterm[2] * dot3(dA + 6, S);
                        }
                        /* d log(F_latt^2) / d N_a */
                        for (int a = 0; a < 3; ++a)
                            dacc[6 + a] += term * (2.0 / N[a] - 4.0 * N[a] *
                                                   fr[a] * fr[a] / 0.63);
                        if (gF) {
                            /* F_cell is linear in the table entries */
                            for (int t = 0; t < nlin; ++t)
                                gF[lin_i[t]] += w_p * Kc * p->scale * 2.0 *
                                                Fc * Fl * Fl * wfac * lin_c[t];
                        }
                    }
                }
            }
    for (int r = 0; r < 9; ++r)
        g[r] += w_p * Kc * p->scale * dacc[r];
    g[9] += w_p * I / p->scale;
}

/* Poisson loss over the pixels pix[0..n) against the target y (bkg added
 * to the model) and its gradient.  p->axes is overwritten from (U, cell,
 * rot).  Gaussian shape only (else returns -3); nearest or tricubic
 * lookup.  grad: 10 values (tx, ty, tz, a, b, c, Na, Nb, Nc, scale); gradF: one
 * value per table entry (may be NULL); model: receives I_p (n values). */
int orc_loss_grad(orc_params *p, const double *U, const double *cell,
                  const double *rot, const long long *pix, long long n,
                  const double *y, double bkg, double *loss, double *grad,
                  double *gradF, double *model, int nthreads)
{
    if (p->shape != 1)
        return -3;
    double d_axes[6 * 9];
    orc_param_axes(U, cell, rot, p->axes, d_axes);
    int PM = p->n_phi * p->n_mosaic;
    double *ax = (double *)malloc((size_t)PM * 9 * sizeof(double));
    double *dax = (double *)malloc((size_t)PM * 6 * 9 * sizeof(double));
    double *tmp = (double *)malloc((size_t)PM * 9 * sizeof(double));
    if (!ax || !dax || !tmp) {
        free(ax);
        free(dax);
        free(tmp);
        return -2;
    }
    rotated_axes(p, ax);
    /* the phi and mosaic rotations are linear maps of the lab axes, so the
     * derivative of every rotated axis is the rotated derivative */
    orc_params q = *p;
    for (int r = 0; r < 6; ++r) {
        memcpy(q.axes, d_axes + 9 * r, sizeof q.axes);
        rotated_axes(&q, tmp);
        for (int jm = 0; jm < PM; ++jm)
            memcpy(dax + ((size_t)jm * 6 + r) * 9, tmp + (size_t)jm * 9,
                   9 * sizeof(double));
    }
    free(tmp);
    size_t nF = (size_t)p->hkl_n[0] * p->hkl_n[1] * p->hkl_n[2];
    if (gradF)
        memset(gradF, 0, nF * sizeof(double));
    double g[10] = {0}, L = 0.0;
    int bad = 0;
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        double gl[10] = {0}, Ll = 0.0;
        double *gF = gradF ? (double *)calloc(nF, sizeof(double)) : NULL;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 8) reduction(| : bad)
#endif
        for (long long ii = 0; ii < n; ++ii) {
            int qq;
            long s, f;
            locate(p, pix[ii], &qq, &s, &f);
            if (qq < 0) {
                bad = 1;
                continue;
            }
            double I = pixel_value(p, ax, qq, s, f);
            model[ii] = I;
            Ll += (I + bkg) - y[ii] * log(I + bkg);
            pixel_grad(p, ax, dax, qq, s, f, I, 1.0 - y[ii] / (I + bkg), gl,
                       gF);
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            for (int r = 0; r < 10; ++r)
                g[r] += gl[r];
            L += Ll;
            if (gF)
                for (size_t e = 0; e < nF; ++e)
                    gradF[e] += gF[e];
        }
        free(gF);
    }
    free(ax);
    free(dax);
    if (bad)
        return -1;
    *loss = L;
    memcpy(grad, g, sizeof g);
    return 0;
}
