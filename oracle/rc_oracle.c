/* rc_oracle.c - plain FP64 CPU oracle of one particle region-competition iteration
 * with particle-approximated Sobolev gradients (arXiv:1403.0240).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path. Slow on purpose: every
 * step follows the paper (or the reading stated where the paper is silent) in the
 * plainest form, in ascending particle-key order (pixel index, then candidate
 * label). Build with -ffp-contract=off so that no multiply-add is fused.
 *
 * Readings where the paper is silent (the optimizer's details are deferred to
 * Cardinale et al. 2012, which is not available):
 *  - A particle is a pair (pixel x, candidate label c) where L(x) != c and some
 *    connectivity-neighbour of x has label c: particles sit on both sides of the
 *    contour (Fig. 1, "Discrete particle approximation").
 *  - Piecewise-constant data term: sum of squared deviations from the region means
 *    (theta_i = region mean, Methods "Bayesian image models"); the energy change of
 *    one flip is the exact single-pixel SSE change.
 *  - Piecewise-smooth data term: local means over a ball of radius R.
 *  - Deconvolving data term (Eq. 8): sum (I - K * s_theta)^2 with theta the region means,
 *    K a separable symmetric PSF, zero outside the image; a flip is evaluated with theta
 *    held (the change of s is at the flipped pixel only).
 *  - Length prior: number of connectivity-adjacent pixel pairs with different labels.
 *  - Eq. 6 sets use the strict cutoff d < E/2, are normalised by their counts, and an
 *    empty set contributes 0; every q uses its pre-update energy difference.
 *  - Ranking before the moves ("The Region Competition (RC) algorithm"): per pixel
 *    the smallest (g, c) is its candidate if g < 0; candidates that keep every
 *    foreground region's topology (simple points) are accepted greedily in
 *    ascending (g, pixel) order, skipping any within Chebyshev distance 1 of an
 *    accepted pixel.
 *  - Oscillation fallback (Eq. 6 discussion): switch to L2 for good once the
 *    accepted-move count has not reached a new minimum for osc_window iterations;
 *    an L2 iteration with no accepted move means convergence.
 */
#include "rc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Eq. 5: K(r) = (1/E) (1 + ((|r|/E)^2 - |r|/E + 1/6) / (2 eps)), |r| <= E/2 */
double orc_kernel_eq5(double r, double E, double eps)
{
    double x = fabs(r) / E;
    double num = x * x - x + 1.0 / 6.0;
    return (1.0 / E) * (1.0 + num / (2.0 * eps));
}

double orc_log(double x)
{
    int e = 0;
    double m = frexp(x, &e);                 /* x = m 2^e, m in [1/2, 1) */
    if (m < 0.70710678118654752440) { m = 2.0 * m; e = e - 1; }
    double y = (m - 1.0) / (m + 1.0);
    double y2 = y * y;
    double s = 1.0 / 23.0;
    s = 1.0 / 21.0 + y2 * s;
    s = 1.0 / 19.0 + y2 * s;
    s = 1.0 / 17.0 + y2 * s;
    s = 1.0 / 15.0 + y2 * s;
    s = 1.0 / 13.0 + y2 * s;
    s = 1.0 / 11.0 + y2 * s;
    s = 1.0 / 9.0 + y2 * s;
    s = 1.0 / 7.0 + y2 * s;
    s = 1.0 / 5.0 + y2 * s;
    s = 1.0 / 3.0 + y2 * s;
    s = 1.0 + y2 * s;
    return (double)e * 0.69314718055994530942 + 2.0 * (y * s);
}

/* Poisson negative log-likelihood of intensity v under mean mu (the log(v!) term dropped),
 * the mean floored at mu_floor */
static double poisson_f(double v, double mu, double mu_floor)
{
    double m = mu > mu_floor ? mu : mu_floor;
    return m - v * orc_log(m);
}

/* ------------------------------------------------------------------ */
static double pix(const orc_params* p, const void* I, int64_t i)
{
    if (p->dtype == 0) return (double)((const float*)I)[i];
    return (double)((const uint16_t*)I)[i];
}

static void coords(const orc_params* p, int64_t i, int64_t* z, int64_t* y, int64_t* x)
{
    *x = i % p->W;
    *y = (i / p->W) % p->H;
    *z = i / (p->W * p->H);
}

static int inside(const orc_params* p, int64_t z, int64_t y, int64_t x)
{
    return z >= 0 && z < p->D && y >= 0 && y < p->H && x >= 0 && x < p->W;
}

/* connectivity neighbours: 4 in 2D, 6 in 3D */
static int nbr_offsets(const orc_params* p, int off[6][3])
{
    int k = 0;
    if (p->ndim == 3) {
        off[k][0] = -1; off[k][1] = 0; off[k][2] = 0; k++;
        off[k][0] = 1;  off[k][1] = 0; off[k][2] = 0; k++;
    }
    off[k][0] = 0; off[k][1] = -1; off[k][2] = 0; k++;
    off[k][0] = 0; off[k][1] = 1;  off[k][2] = 0; k++;
    off[k][0] = 0; off[k][1] = 0;  off[k][2] = -1; k++;
    off[k][0] = 0; off[k][1] = 0;  off[k][2] = 1; k++;
    return k;
}

/* ------------------------------------------------------------------ */
/* Particles: every (x, c) with c != L(x) the label of a connectivity neighbour. */
int64_t orc_extract(const orc_params* p, const int32_t* L,
                    uint32_t* idx, int32_t* l, int32_t* c, int64_t cap)
{
    int off[6][3];
    int nn = nbr_offsets(p, off);
    int64_t npix = p->D * p->H * p->W;
    int64_t count = 0;
    for (int64_t i = 0; i < npix; i++) {
        int64_t z, y, x;
        coords(p, i, &z, &y, &x);
        int32_t own = L[i];
        int32_t labs[6];
        int nl = 0;
        for (int k = 0; k < nn; k++) {
            int64_t zz = z + off[k][0], yy = y + off[k][1], xx = x + off[k][2];
            if (!inside(p, zz, yy, xx)) continue;
            int32_t m = L[(zz * p->H + yy) * p->W + xx];
            if (m == own) continue;
            int seen = 0;
            for (int j = 0; j < nl; j++) if (labs[j] == m) seen = 1;
            if (!seen) labs[nl++] = m;
        }
        /* ascending candidate label */
        for (int a = 1; a < nl; a++)
            for (int b = a; b > 0 && labs[b - 1] > labs[b]; b--) {
                int32_t t = labs[b]; labs[b] = labs[b - 1]; labs[b - 1] = t;
            }
        for (int j = 0; j < nl; j++) {
            if (count < cap) {
                idx[count] = (uint32_t)i;
                l[count] = own;
                c[count] = labs[j];
            }
            count++;
        }
    }
    return count;
}

/* ------------------------------------------------------------------ */
/* Exact summation: a big fixed-point integer with least significant bit 2^-300,
 * 32 value bits per limb; positive and negative parts kept apart, rounded once
 * to the nearest double (ties to even). */
#define ACC_LIMBS 24
#define ACC_LSB (-300)

typedef struct { uint64_t pos[ACC_LIMBS], neg[ACC_LIMBS]; int64_t adds; } bigacc;

static void acc_norm(uint64_t* a)
{
    uint64_t carry = 0;
    for (int k = 0; k < ACC_LIMBS; k++) {
        uint64_t t = a[k] + carry;
        a[k] = t & 0xFFFFFFFFull;
        carry = t >> 32;
    }
}

/* add m * 2^(s + ACC_LSB), m < 2^49, s >= 0 */
static void acc_add(bigacc* A, int neg, uint64_t m, int s)
{
    uint64_t* a = neg ? A->neg : A->pos;
    int k = s / 32, r = s % 32;
    /* m * 2^r has at most 81 bits: bits 0-31, 32-63 and 64-95 go to limbs k, k+1, k+2 */
    uint64_t lo = (m << r) & 0xFFFFFFFFull;
    uint64_t mid, hi;
    if (r == 0) {
        mid = (m >> 32) & 0xFFFFFFFFull;
        hi = 0;
    } else {
        mid = (m >> (32 - r)) & 0xFFFFFFFFull;
        hi = m >> (64 - r);
    }
    a[k] += lo;
    if (k + 1 < ACC_LIMBS) a[k + 1] += mid;
    if (k + 2 < ACC_LIMBS) a[k + 2] += hi;
    if (++A->adds >= (1 << 24)) { acc_norm(A->pos); acc_norm(A->neg); A->adds = 0; }
}

static void acc_add_f32(bigacc* A, float f, int squares)
{
    uint32_t bits;
    memcpy(&bits, &f, 4);
    int sign = (int)(bits >> 31);
    int eb = (int)((bits >> 23) & 0xFF);
    uint64_t m = bits & 0x7FFFFFu;
    if (eb == 0) eb = 1; else m |= 0x800000u;   /* subnormals share the smallest scale */
    if (m == 0) return;
    /* |f| = m * 2^(eb - 150) */
    if (!squares) acc_add(A, sign, m, eb - 150 - ACC_LSB);
    else acc_add(A, 0, m * m, 2 * (eb - 150) - ACC_LSB);
}

static void acc_add_int(bigacc* A, uint64_t m)
{
    if (m) acc_add(A, 0, m, -ACC_LSB);
}

static int big_cmp(const uint64_t* a, const uint64_t* b)
{
    for (int k = ACC_LIMBS - 1; k >= 0; k--) {
        if (a[k] != b[k]) return a[k] > b[k] ? 1 : -1;
    }
    return 0;
}

static void big_sub(uint64_t* r, const uint64_t* a, const uint64_t* b)  /* r = a - b, a >= b */
{
    int64_t borrow = 0;
    for (int k = 0; k < ACC_LIMBS; k++) {
        int64_t t = (int64_t)a[k] - (int64_t)b[k] - borrow;
        borrow = t < 0;
        if (t < 0) t += (int64_t)1 << 32;
        r[k] = (uint64_t)t;
    }
}

static int big_bit(const uint64_t* a, int b) { return (int)((a[b / 32] >> (b % 32)) & 1u); }

static double acc_round(bigacc* A)
{
    acc_norm(A->pos);
    acc_norm(A->neg);
    uint64_t mag[ACC_LIMBS];
    int sign = 0;
    int cmp = big_cmp(A->pos, A->neg);
    if (cmp == 0) return 0.0;
    if (cmp > 0) big_sub(mag, A->pos, A->neg);
    else { big_sub(mag, A->neg, A->pos); sign = 1; }
    int h = -1;
    for (int b = ACC_LIMBS * 32 - 1; b >= 0; b--) if (big_bit(mag, b)) { h = b; break; }
    uint64_t mant = 0;
    int shift = 0;
    if (h <= 52) {
        for (int b = h; b >= 0; b--) mant = (mant << 1) | (uint64_t)big_bit(mag, b);
    } else {
        shift = h - 52;
        for (int b = h; b >= shift; b--) mant = (mant << 1) | (uint64_t)big_bit(mag, b);
        int round = big_bit(mag, shift - 1);
        int sticky = 0;
        for (int b = shift - 2; b >= 0; b--) if (big_bit(mag, b)) { sticky = 1; break; }
        if (round && (sticky || (mant & 1u))) {
            mant++;
            if (mant == (1ull << 53)) { mant >>= 1; shift++; }
        }
    }
    double v = ldexp((double)mant, shift + ACC_LSB);
    return sign ? -v : v;
}

double orc_exact_sum_f32(const float* v, int64_t n, int squares)
{
    bigacc A;
    memset(&A, 0, sizeof A);
    for (int64_t i = 0; i < n; i++) acc_add_f32(&A, v[i], squares);
    return acc_round(&A);
}

/* Region statistics: n_i = |Omega_i|, S_i = sum I, Q_i = sum I^2, each exact and
 * rounded once (theta_i = S_i / n_i is the region mean, Methods). */
void orc_stats(const orc_params* p, const void* I, const int32_t* L,
               int64_t* n, double* S, double* Q)
{
    int M = p->nlabels;
    bigacc* AS = (bigacc*)calloc((size_t)M, sizeof(bigacc));
    bigacc* AQ = (bigacc*)calloc((size_t)M, sizeof(bigacc));
    int64_t npix = p->D * p->H * p->W;
    for (int m = 0; m < M; m++) n[m] = 0;
    for (int64_t i = 0; i < npix; i++) {
        int32_t m = L[i];
        n[m]++;
        if (p->dtype == 0) {
            float f = ((const float*)I)[i];
            acc_add_f32(&AS[m], f, 0);
            acc_add_f32(&AQ[m], f, 1);
        } else {
            uint64_t u = ((const uint16_t*)I)[i];
            acc_add_int(&AS[m], u);
            acc_add_int(&AQ[m], u * u);
        }
    }
    for (int m = 0; m < M; m++) {
        S[m] = acc_round(&AS[m]);
        Q[m] = acc_round(&AQ[m]);
    }
    free(AS);
    free(AQ);
}

/* ------------------------------------------------------------------ */
/* Deconvolving model (Eq. 8): the expected image is J = s_theta(Gamma) * K, s_theta the
 * piecewise-constant image-generating function (theta_i the region means, the usual estimate
 * named with Eq. 7), K the PSF, zero outside the image. The data term is sum_x (I - J)^2. */

/* one axis of the separable correlation: out(x) = sum_u k(u) f(x + u e_axis) */
static void psf_axis(const orc_params* p, const double* f, double* out, int axis)
{
    int r = p->psf_r;
    int64_t extent[3] = {p->W, p->H, p->D};
    int64_t stride[3] = {1, p->W, p->W * p->H};
    int64_t npix = p->D * p->H * p->W;
    for (int64_t i = 0; i < npix; i++) {
        int64_t z, y, x;
        coords(p, i, &z, &y, &x);
        int64_t t = axis == 0 ? x : (axis == 1 ? y : z);
        double acc = 0.0;
        for (int u = -r; u <= r; u++) {
            if (t + u < 0 || t + u >= extent[axis]) continue;   /* f = 0 outside */
            acc = fma(p->psf[u + r], f[i + u * stride[axis]], acc);
        }
        out[i] = acc;
    }
}

void orc_psf_correlate(const orc_params* p, const double* f, double* out)
{
    int64_t npix = p->D * p->H * p->W;
    double* t = (double*)malloc(sizeof(double) * (size_t)(npix > 0 ? npix : 1));
    psf_axis(p, f, t, 0);
    if (p->ndim == 3) {
        double* t2 = (double*)malloc(sizeof(double) * (size_t)(npix > 0 ? npix : 1));
        psf_axis(p, t, t2, 1);
        psf_axis(p, t2, out, 2);
        free(t2);
    } else {
        psf_axis(p, t, out, 1);
    }
    free(t);
}

void orc_deconv_fields(const orc_params* p, const void* I, const int32_t* L,
                       const int64_t* n, const double* S, double* J, double* R, double* G)
{
    int64_t npix = p->D * p->H * p->W;
    size_t nb = sizeof(double) * (size_t)(npix > 0 ? npix : 1);
    double* s = (double*)malloc(nb);
    double* j = (double*)malloc(nb);
    double* r = (double*)malloc(nb);
    for (int64_t i = 0; i < npix; i++) {
        int32_t m = L[i];
        s[i] = n[m] > 0 ? S[m] / (double)n[m] : 0.0;
    }
    orc_psf_correlate(p, s, j);
    for (int64_t i = 0; i < npix; i++) r[i] = pix(p, I, i) - j[i];
    orc_psf_correlate(p, r, G);
    if (J) memcpy(J, j, nb);
    if (R) memcpy(R, r, nb);
    free(s);
    free(j);
    free(r);
}

static double psf_norm2_axis(const orc_params* p, int64_t t, int64_t extent)
{
    int r = p->psf_r;
    double acc = 0.0;
    for (int u = -r; u <= r; u++) {
        if (t + u < 0 || t + u >= extent) continue;
        acc = fma(p->psf[u + r], p->psf[u + r], acc);
    }
    return acc;
}

double orc_psf_norm2(const orc_params* p, int64_t z, int64_t y, int64_t x)
{
    double v = psf_norm2_axis(p, x, p->W) * psf_norm2_axis(p, y, p->H);
    if (p->ndim == 3) v = v * psf_norm2_axis(p, z, p->D);
    return v;
}

/* ------------------------------------------------------------------ */
/* Length prior: change of the number of connectivity-adjacent pixel pairs with
 * different labels when x goes from l to c (neighbours outside the image absent). */
int64_t orc_delta_perimeter(const orc_params* p, const int32_t* L, uint32_t xi, int32_t l, int32_t c)
{
    int off[6][3];
    int nn = nbr_offsets(p, off);
    int64_t z, y, x;
    coords(p, xi, &z, &y, &x);
    int64_t d = 0;
    for (int k = 0; k < nn; k++) {
        int64_t zz = z + off[k][0], yy = y + off[k][1], xx = x + off[k][2];
        if (!inside(p, zz, yy, xx)) continue;
        int32_t m = L[(zz * p->H + yy) * p->W + xx];
        d += (int64_t)(m != c) - (int64_t)(m != l);
    }
    return d;
}

/* Length of the contour |Gamma| in the discrete reading used by the length prior: the
 * number of connectivity-adjacent pixel pairs with different labels (each pair once). */
int64_t orc_perimeter(const orc_params* p, const int32_t* L)
{
    int64_t P = 0;
    for (int64_t z = 0; z < p->D; z++)
        for (int64_t y = 0; y < p->H; y++)
            for (int64_t x = 0; x < p->W; x++) {
                int32_t m = L[(z * p->H + y) * p->W + x];
                if (x + 1 < p->W && L[(z * p->H + y) * p->W + x + 1] != m) P++;
                if (y + 1 < p->H && L[(z * p->H + y + 1) * p->W + x] != m) P++;
                if (p->ndim == 3 && z + 1 < p->D && L[((z + 1) * p->H + y) * p->W + x] != m) P++;
            }
    return P;
}

/* ------------------------------------------------------------------ */
/* Curvature regulariser (reading of the curvature regularisation used with weight lambda in the
 * experiments; RC estimates curvature by counting pixels in a sphere around x). Integral
 * invariants (Pottmann et al. 2007): a ball of radius rho centred on the boundary of a region
 * holds A = (pi/2) rho^2 - (kappa/3) rho^3 + O(rho^4) of it in 2D, and
 * V = (2 pi/3) rho^3 - (pi/4) H rho^4 + O(rho^5) in 3D, H = (kappa_1 + kappa_2)/2 the mean
 * curvature. With A_m(x) the ball's pixels of label m this gives kappa_m = 3 ((pi/2) rho^2 - A_m)
 * / rho^3 and kappa_1 + kappa_2 = 2 H_m = 8 ((2 pi/3) rho^3 - V_m) / (pi rho^4). Moving x from l to
 * c shrinks l and grows c by one pixel; the first variation of a boundary's length (area) under
 * a normal displacement of unit area (volume) is its curvature (kappa_1 + kappa_2), and every
 * interface bounds two regions, so |Gamma| = (1/2) sum_m |boundary of m| changes by half the
 * difference of the two curvatures. The constant terms cancel, leaving w (A_l - A_c) with
 * w = lambda * 3 / (2 rho^3) (2D) and lambda * 4 / (pi rho^4) (3D). */
int64_t orc_ball_balance(const orc_params* p, const int32_t* L, uint32_t xi, int32_t l, int32_t c)
{
    int Ri = (int)floor(p->curv_radius);
    double R2 = p->curv_radius * p->curv_radius;
    int Rz = p->ndim == 3 ? Ri : 0;
    int64_t z, y, x;
    coords(p, xi, &z, &y, &x);
    int64_t bal = 0;
    for (int dz = -Rz; dz <= Rz; dz++)
        for (int dy = -Ri; dy <= Ri; dy++)
            for (int dx = -Ri; dx <= Ri; dx++) {
                int64_t d2 = (int64_t)dz * dz + (int64_t)dy * dy + (int64_t)dx * dx;
                if (!((double)d2 <= R2)) continue;
                int64_t zz = z + dz, yy = y + dy, xx = x + dx;
                if (!inside(p, zz, yy, xx)) continue;
                int32_t m = L[(zz * p->H + yy) * p->W + xx];
                if (m == l) bal++;
                else if (m == c) bal--;
            }
    return bal;
}

/* the weight, evaluated as written (products and one quotient, no sum) */
double orc_curvature_weight(const orc_params* p)
{
    double r = p->curv_radius;
    if (p->ndim == 3) return p->lambda * (4.0 / (3.141592653589793 * (r * r * r * r)));
    return p->lambda * (3.0 / (2.0 * (r * r * r)));
}

/* Energy difference of moving particle (x: l -> c), data term + regulariser (lambda * change
 * of the contour length, or the curvature term above). */
void orc_energy(const orc_params* p, const void* I, const int32_t* L,
                const int64_t* n, const double* S, int64_t N,
                const uint32_t* idx, const int32_t* l, const int32_t* c, double* dE, double* scale)
{
    int Ri = (int)floor(p->ps_radius);
    double R2 = p->ps_radius * p->ps_radius;
    double* G = NULL;
    if (p->model == 3) {
        int64_t npix = p->D * p->H * p->W;
        G = (double*)malloc(sizeof(double) * (size_t)(npix > 0 ? npix : 1));
        orc_deconv_fields(p, I, L, n, S, NULL, NULL, G);
    }
    for (int64_t k = 0; k < N; k++) {
        uint32_t xi = idx[k];
        int32_t lp = l[k], cp = c[k];
        double v = pix(p, I, xi);
        double data;
        if (p->model == 3) {
            /* Deconvolving: with theta held, moving x from l to c adds d K(. - x) to J, so the
             * data term changes by sum (R - d K_x)^2 - R^2 = d^2 |K_x|^2 - 2 d (K * R)(x). */
            int64_t z, y, x;
            coords(p, xi, &z, &y, &x);
            double thc = n[cp] > 0 ? S[cp] / (double)n[cp] : 0.0;
            double thl = n[lp] > 0 ? S[lp] / (double)n[lp] : 0.0;
            double d = thc - thl;
            double t = d * G[xi];
            double q = (d * d) * orc_psf_norm2(p, z, y, x);
            data = q - (t + t);
            if (scale) scale[k] = fabs(q) + fabs(t + t);
        } else if (p->model == 0) {
            /* Piecewise constant: exact SSE change of moving v from region l to c. */
            double mc = S[cp] / (double)n[cp];
            double ml = S[lp] / (double)n[lp];
            double a = v - mc;
            double b = v - ml;
            double t1 = ((double)n[cp] / ((double)n[cp] + 1.0)) * (a * a);
            double t2 = 0.0;
            if (n[lp] > 1) t2 = ((double)n[lp] / ((double)n[lp] - 1.0)) * (b * b);
            data = t1 - t2;
            if (scale) scale[k] = fabs(t1) + fabs(t2);
        } else {
            /* Piecewise smooth: local means over the ball of radius R, row-major order. */
            int64_t z, y, x;
            coords(p, xi, &z, &y, &x);
            double sc = 0.0, sl = 0.0;
            int64_t cc = 0, cl = 0;
            int Rz = p->ndim == 3 ? Ri : 0;
            for (int dz = -Rz; dz <= Rz; dz++)
                for (int dy = -Ri; dy <= Ri; dy++)
                    for (int dx = -Ri; dx <= Ri; dx++) {
                        int64_t d2 = (int64_t)dz * dz + (int64_t)dy * dy + (int64_t)dx * dx;
                        if (!((double)d2 <= R2)) continue;
                        int64_t zz = z + dz, yy = y + dy, xx = x + dx;
                        if (!inside(p, zz, yy, xx)) continue;
                        int64_t j = (zz * p->H + yy) * p->W + xx;
                        int32_t m = L[j];
                        if (m == cp) { sc = sc + pix(p, I, j); cc++; }
                        else if (m == lp) { sl = sl + pix(p, I, j); cl++; }
                    }
            double muc = sc / (double)cc;
            double mul = sl / (double)cl;
            if (p->model == 2) {
                /* Poisson noise: -log p(v | mu) = mu - v ln mu, the local means as the model */
                double fc = poisson_f(v, muc, p->mu_floor);
                double fl = poisson_f(v, mul, p->mu_floor);
                data = fc - fl;
                if (scale) {
                    /* the four terms of (m_c - v ln m_c) - (m_l - v ln m_l), means floored */
                    double mc = muc > p->mu_floor ? muc : p->mu_floor;
                    double ml = mul > p->mu_floor ? mul : p->mu_floor;
                    scale[k] = fabs(mc) + fabs(v * orc_log(mc)) + fabs(ml) + fabs(v * orc_log(ml));
                }
            } else {
                double a = v - muc;
                double b = v - mul;
                data = a * a - b * b;
                if (scale) scale[k] = a * a + b * b;
            }
        }
        int64_t dP;
        double w;
        if (p->regulariser == 1) {
            dP = orc_ball_balance(p, L, xi, lp, cp);
            w = orc_curvature_weight(p);
        } else {
            dP = orc_delta_perimeter(p, L, xi, lp, cp);
            w = p->lambda;
        }
        dE[k] = data + w * (double)dP;
        if (scale) scale[k] += fabs(w * (double)dP);
    }
    free(G);
}

/* ------------------------------------------------------------------ */
/* Eq. 6 on particles, neighbours found with a cell list of edge ceil(E/2). */
static int cmp_i64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

void orc_sobolev(const orc_params* p, int64_t N, const uint32_t* idx, const int32_t* l,
                 const int32_t* c, const double* dE, int all_pairs,
                 double* g, double* A, double* B, int32_t* nQ, int32_t* nQp, double* scale)
{
    double rc = p->cutoff;
    double r2 = rc * rc;
    double E = 2.0 * rc;
    double eps = 1.0 / 24.0;
    int64_t s = (int64_t)ceil(rc);
    if (s < 1) s = 1;
    int64_t ncx = (p->W + s - 1) / s, ncy = (p->H + s - 1) / s, ncz = (p->D + s - 1) / s;
    int64_t ncell = ncx * ncy * ncz;
    int64_t* cz = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int64_t* cy = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int64_t* cx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int64_t* cstart = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int64_t* fill = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t k = 0; k < N; k++) {
        coords(p, idx[k], &cz[k], &cy[k], &cx[k]);
        int64_t cell = ((cz[k] / s) * ncy + cy[k] / s) * ncx + cx[k] / s;
        cstart[cell + 1]++;
    }
    for (int64_t q = 0; q < ncell; q++) cstart[q + 1] += cstart[q];
    for (int64_t k = 0; k < N; k++) {
        int64_t cell = ((cz[k] / s) * ncy + cy[k] / s) * ncx + cx[k] / s;
        order[cstart[cell] + fill[cell]++] = k;
    }
    for (int64_t k = 0; k < N; k++) {
        int64_t nlist = 0;
        if (all_pairs) {
            for (int64_t q = 0; q < N; q++) list[nlist++] = q;
        } else {
            int64_t kz = cz[k] / s, ky = cy[k] / s, kx = cx[k] / s;
            for (int64_t dz = -1; dz <= 1; dz++)
                for (int64_t dy = -1; dy <= 1; dy++)
                    for (int64_t dx = -1; dx <= 1; dx++) {
                        int64_t zz = kz + dz, yy = ky + dy, xx = kx + dx;
                        if (zz < 0 || zz >= ncz || yy < 0 || yy >= ncy || xx < 0 || xx >= ncx) continue;
                        int64_t cell = (zz * ncy + yy) * ncx + xx;
                        for (int64_t j = cstart[cell]; j < cstart[cell + 1]; j++) {
                            int64_t q = order[j];
                            int64_t ez = cz[q] - cz[k], ey = cy[q] - cy[k], ex = cx[q] - cx[k];
                            /* only the particles inside the cutoff take part in the sums */
                            if ((double)(ez * ez + ey * ey + ex * ex) < r2) list[nlist++] = q;
                        }
                    }
            qsort(list, (size_t)nlist, sizeof(int64_t), cmp_i64);   /* ascending particle key */
        }
        double As = 0.0, Bs = 0.0, Aa = 0.0, Ba = 0.0;
        int32_t na = 0, nb = 0;
        for (int64_t t = 0; t < nlist; t++) {
            int64_t q = list[t];
            int64_t ddz = cz[q] - cz[k], ddy = cy[q] - cy[k], ddx = cx[q] - cx[k];
            int64_t d2 = ddz * ddz + ddy * ddy + ddx * ddx;
            if (!((double)d2 < r2)) continue;
            double K = orc_kernel_eq5(sqrt((double)d2), E, eps);
            if (l[q] == l[k]) { As = As + K * dE[q]; Aa += fabs(K * dE[q]); na++; }
            if (c[q] == l[k]) { Bs = Bs + K * dE[q]; Ba += fabs(K * dE[q]); nb++; }
        }
        double a = na ? As / (double)na : 0.0;
        double b = nb ? Bs / (double)nb : 0.0;
        g[k] = a - b;
        if (A) A[k] = a;
        if (B) B[k] = b;
        if (nQ) nQ[k] = na;
        if (nQp) nQp[k] = nb;
        if (scale) scale[k] = (na ? Aa / (double)na : 0.0) + (nb ? Ba / (double)nb : 0.0);
    }
    free(cz); free(cy); free(cx); free(cstart); free(order); free(fill); free(list);
}

/* ------------------------------------------------------------------ */
/* Simple points by topological numbers (Bertrand & Malandain 1994).
 * 2D, foreground 4 / background 8: T4 = number of 4-components of X in the
 * 8-neighbourhood that contain a 4-neighbour of x; T8 = number of 8-components of
 * the complement in the 8-neighbourhood. 3D, foreground 6 / background 26: T6 =
 * number of 6-components of X in the 18-neighbourhood containing a 6-neighbour of
 * x; T26 = number of 26-components of the complement in the 26-neighbourhood.
 * x is simple iff both numbers are 1. Components are found by breadth-first
 * search over the window cells. */
static int count_components(int ncell, const int* member, const int (*pos)[3],
                            int adjacency, const int* must_touch)
{
    int label[27];
    int queue[27];
    for (int i = 0; i < ncell; i++) label[i] = -1;
    int ncomp = 0, counted = 0;
    for (int s0 = 0; s0 < ncell; s0++) {
        if (!member[s0] || label[s0] >= 0) continue;
        int head = 0, tail = 0, touches = 0;
        queue[tail++] = s0;
        label[s0] = ncomp;
        while (head < tail) {
            int u = queue[head++];
            if (must_touch && must_touch[u]) touches = 1;
            for (int v = 0; v < ncell; v++) {
                if (!member[v] || label[v] >= 0) continue;
                int dz = abs(pos[u][0] - pos[v][0]), dy = abs(pos[u][1] - pos[v][1]), dx = abs(pos[u][2] - pos[v][2]);
                int l1 = dz + dy + dx, linf = dz > dy ? (dz > dx ? dz : dx) : (dy > dx ? dy : dx);
                int adj = adjacency == 6 || adjacency == 4 ? (l1 == 1) : (linf == 1);
                if (adj) { label[v] = ncomp; queue[tail++] = v; }
            }
        }
        ncomp++;
        if (!must_touch || touches) counted++;
    }
    return counted;
}

int orc_simple_2d(const uint8_t* nb9)
{
    int pos[8][3], fg[8], bg[8], touch[8];
    int k = 0;
    for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
            if (dy == 0 && dx == 0) continue;
            pos[k][0] = 0; pos[k][1] = dy; pos[k][2] = dx;
            int in = nb9[(dy + 1) * 3 + (dx + 1)] != 0;
            fg[k] = in;
            bg[k] = !in;
            touch[k] = (abs(dy) + abs(dx)) == 1;
            k++;
        }
    int t4 = count_components(8, fg, (const int (*)[3])pos, 4, touch);
    int t8 = count_components(8, bg, (const int (*)[3])pos, 8, NULL);
    return t4 == 1 && t8 == 1;
}

int orc_simple_3d(const uint8_t* nb27)
{
    int pos[26][3], fg18[26], bg[26], touch[26];
    int k = 0;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                if (dz == 0 && dy == 0 && dx == 0) continue;
                pos[k][0] = dz; pos[k][1] = dy; pos[k][2] = dx;
                int in = nb27[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] != 0;
                int l1 = abs(dz) + abs(dy) + abs(dx);
                fg18[k] = in && l1 <= 2;
                bg[k] = !in;
                touch[k] = l1 == 1;
                k++;
            }
    int t6 = count_components(26, fg18, (const int (*)[3])pos, 6, touch);
    int t26 = count_components(26, bg, (const int (*)[3])pos, 26, NULL);
    return t6 == 1 && t26 == 1;
}

static int simple_for_label(const orc_params* p, const int32_t* L, uint32_t xi, int32_t lab)
{
    int64_t z, y, x;
    coords(p, xi, &z, &y, &x);
    uint8_t nb[27];
    int k = 0;
    int rz = p->ndim == 3 ? 1 : 0;
    for (int dz = -rz; dz <= rz; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int64_t zz = z + dz, yy = y + dy, xx = x + dx;
                int in = 0;
                if (inside(p, zz, yy, xx)) in = L[(zz * p->H + yy) * p->W + xx] == lab;
                nb[k++] = (uint8_t)in;
            }
    return p->ndim == 3 ? orc_simple_3d(nb) : orc_simple_2d(nb);
}

/* Region vanishing: x is the last pixel of its region exactly when no connectivity neighbour
 * of x has its label (every foreground label is one connected component). */
static int last_pixel_of(const orc_params* p, const int32_t* L, uint32_t xi, int32_t lab)
{
    int off[6][3];
    int n = nbr_offsets(p, off);
    int64_t z, y, x;
    coords(p, xi, &z, &y, &x);
    for (int k = 0; k < n; k++) {
        int64_t zz = z + off[k][0], yy = y + off[k][1], xx = x + off[k][2];
        if (inside(p, zz, yy, xx) && L[(zz * p->H + yy) * p->W + xx] == lab) return 0;
    }
    return 1;
}

/* Foreground topological number of x for label lab: connectivity components of the label's
 * pixels in the neighbourhood (the 8-neighbourhood in 2D, the 18-neighbourhood in 3D) that
 * contain a connectivity neighbour of x. */
static int foreground_number(const orc_params* p, const int32_t* L, uint32_t xi, int32_t lab)
{
    int64_t z, y, x;
    coords(p, xi, &z, &y, &x);
    int pos[26][3], fg[26], touch[26];
    int k = 0;
    int rz = p->ndim == 3 ? 1 : 0;
    for (int dz = -rz; dz <= rz; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                if (dz == 0 && dy == 0 && dx == 0) continue;
                int64_t zz = z + dz, yy = y + dy, xx = x + dx;
                int in = inside(p, zz, yy, xx) && L[(zz * p->H + yy) * p->W + xx] == lab;
                int l1 = abs(dz) + abs(dy) + abs(dx);
                pos[k][0] = dz; pos[k][1] = dy; pos[k][2] = dx;
                fg[k] = in && l1 <= 2;
                touch[k] = l1 == 1;
                k++;
            }
    return count_components(k, fg, (const int (*)[3])pos, p->ndim == 3 ? 6 : 4, touch);
}

/* Topological control: foreground regions stay connected sets without new or lost
 * holes; removal from l (l != 0) and addition to c (c != 0) must both be simple. With
 * topology bit 1 a region may vanish: the removal of its last pixel is admissible too. With
 * bit 2 a removal that locally disconnects the region (foreground number >= 2) is admissible:
 * the region splits, or one of its holes opens to the rest of the image. */
int orc_admissible(const orc_params* p, const int32_t* L, uint32_t xi, int32_t l, int32_t c)
{
    if (l != 0 && !simple_for_label(p, L, xi, l) && !((p->topology & 1) && last_pixel_of(p, L, xi, l)) &&
        !((p->topology & 2) && foreground_number(p, L, xi, l) >= 2))
        return 0;
    if (c != 0 && !simple_for_label(p, L, xi, c)) return 0;
    return 1;
}

/* ------------------------------------------------------------------ */
typedef struct { double g; uint32_t idx; int32_t c; } cand_t;

static int cmp_cand(const void* a, const void* b)
{
    const cand_t* x = (const cand_t*)a;
    const cand_t* y = (const cand_t*)b;
    if (x->g < y->g) return -1;
    if (x->g > y->g) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

int64_t orc_select(const orc_params* p, const int32_t* L, int64_t N,
                   const uint32_t* idx, const int32_t* l, const int32_t* c, const double* g,
                   uint32_t* acc_idx, int32_t* acc_c, int64_t* n_candidates)
{
    cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)(N > 0 ? N : 1));
    int64_t nc = 0;
    int64_t k = 0;
    while (k < N) {
        int64_t e = k;
        while (e < N && idx[e] == idx[k]) e++;
        int64_t best = k;
        for (int64_t j = k + 1; j < e; j++)
            if (g[j] < g[best] || (g[j] == g[best] && c[j] < c[best])) best = j;
        if (g[best] < 0.0 && orc_admissible(p, L, idx[best], l[best], c[best])) {
            cand[nc].g = g[best];
            cand[nc].idx = idx[best];
            cand[nc].c = c[best];
            nc++;
        }
        k = e;
    }
    if (n_candidates) *n_candidates = nc;
    qsort(cand, (size_t)nc, sizeof(cand_t), cmp_cand);
    int64_t npix = p->D * p->H * p->W;
    uint8_t* taken = (uint8_t*)calloc((size_t)npix, 1);
    int64_t na = 0;
    int rz = p->ndim == 3 ? 1 : 0;
    for (int64_t t = 0; t < nc; t++) {
        int64_t z, y, x;
        coords(p, cand[t].idx, &z, &y, &x);
        int blocked = 0;
        for (int dz = -rz; dz <= rz && !blocked; dz++)
            for (int dy = -1; dy <= 1 && !blocked; dy++)
                for (int dx = -1; dx <= 1 && !blocked; dx++) {
                    int64_t zz = z + dz, yy = y + dy, xx = x + dx;
                    if (inside(p, zz, yy, xx) && taken[(zz * p->H + yy) * p->W + xx]) blocked = 1;
                }
        if (blocked) continue;
        taken[cand[t].idx] = 1;
        if (acc_idx) acc_idx[na] = cand[t].idx;
        if (acc_c) acc_c[na] = cand[t].c;
        na++;
    }
    free(taken);
    free(cand);
    return na;
}

/* ------------------------------------------------------------------ */
/* After a split: every foreground label's connectivity components but the one holding its
 * smallest pixel index get new labels, numbered from nlabels upward in ascending order of the
 * components' smallest pixel indices. Components are found by breadth-first search from the
 * pixels in raster order, so each is found at its smallest pixel. Returns the new label count. */
int32_t orc_relabel(const orc_params* p, int32_t* L, int32_t nlabels)
{
    int64_t npix = p->D * p->H * p->W;
    int32_t* comp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(npix > 0 ? npix : 1));
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(npix > 0 ? npix : 1));
    uint8_t* seen_label = (uint8_t*)calloc((size_t)nlabels + 1, 1);
    int off[6][3];
    int nn = nbr_offsets(p, off);
    for (int64_t i = 0; i < npix; i++) comp[i] = 0;
    int32_t next = nlabels;
    for (int64_t s0 = 0; s0 < npix; s0++) {
        int32_t m = L[s0];
        if (m == 0 || comp[s0]) continue;
        int32_t target = m;
        if (m < nlabels && seen_label[m]) target = next++;   /* a further component of m */
        if (m < nlabels) seen_label[m] = 1;
        int64_t head = 0, tail = 0;
        queue[tail++] = s0;
        comp[s0] = 1;
        while (head < tail) {
            int64_t u = queue[head++];
            int64_t z, y, x;
            coords(p, u, &z, &y, &x);
            for (int k = 0; k < nn; k++) {
                int64_t zz = z + off[k][0], yy = y + off[k][1], xx = x + off[k][2];
                if (!inside(p, zz, yy, xx)) continue;
                int64_t v = (zz * p->H + yy) * p->W + xx;
                if (comp[v] || L[v] != m) continue;
                comp[v] = 1;
                queue[tail++] = v;
            }
            L[u] = target;
        }
    }
    free(comp);
    free(queue);
    free(seen_label);
    return next;
}

/* ------------------------------------------------------------------ */
/* Fusion (topology bit 4, piecewise-constant model; reading of RC's controlled merging, whose
 * criterion the paper leaves to its reference): after the moves of an iteration and the
 * relabelling of split pieces, two touching foreground regions a < b fuse when that lowers the
 * energy. Merging them changes the data term by exactly n_a n_b / (n_a + n_b) (mu_a - mu_b)^2
 * (the sum of squared deviations about the joint mean) and removes the B_ab connectivity-
 * adjacent pixel pairs between them from the contour, so
 *     dE = w * (d * d) - lambda * B_ab,  w = (n_a * n_b) / (n_a + n_b),  d = mu_a - mu_b,
 * evaluated in that order with the statistics after the moves. The pairs with dE < 0 are taken
 * in ascending (dE, a, b); a pair is accepted when neither of its labels was accepted before in
 * the iteration, and then b's pixels take label a. Returns the number of fusions. */
typedef struct {
    double dE;
    int32_t a, b;
} fuse_pair;

static int cmp_u64(const void* x, const void* y)
{
    uint64_t a = *(const uint64_t*)x, b = *(const uint64_t*)y;
    return (a > b) - (a < b);
}

static int cmp_fuse(const void* x, const void* y)
{
    const fuse_pair* u = (const fuse_pair*)x;
    const fuse_pair* v = (const fuse_pair*)y;
    if (u->dE != v->dE) return u->dE < v->dE ? -1 : 1;
    if (u->a != v->a) return u->a < v->a ? -1 : 1;
    return (u->b > v->b) - (u->b < v->b);
}

int64_t orc_fuse_pairs(const orc_params* p, const int32_t* L, int32_t* a_out, int32_t* b_out, int64_t* B_out,
                       int64_t cap)
{
    int64_t npix = p->D * p->H * p->W;
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(3 * npix + 1));
    int64_t nk = 0;
    for (int64_t z = 0; z < p->D; z++)
        for (int64_t y = 0; y < p->H; y++)
            for (int64_t x = 0; x < p->W; x++) {
                int64_t i = (z * p->H + y) * p->W + x;
                int32_t m = L[i];
                if (m == 0) continue;
                int64_t nb[3];
                int k = 0;
                if (x + 1 < p->W) nb[k++] = i + 1;
                if (y + 1 < p->H) nb[k++] = i + p->W;
                if (p->ndim == 3 && z + 1 < p->D) nb[k++] = i + p->W * p->H;
                for (int u = 0; u < k; u++) {
                    int32_t m2 = L[nb[u]];
                    if (m2 == 0 || m2 == m) continue;
                    uint32_t a = (uint32_t)(m < m2 ? m : m2), b = (uint32_t)(m < m2 ? m2 : m);
                    keys[nk++] = ((uint64_t)a << 32) | b;
                }
            }
    qsort(keys, (size_t)nk, sizeof(uint64_t), cmp_u64);
    int64_t np = 0;
    for (int64_t i = 0; i < nk;) {
        int64_t j = i;
        while (j < nk && keys[j] == keys[i]) j++;
        if (np < cap) {
            a_out[np] = (int32_t)(keys[i] >> 32);
            b_out[np] = (int32_t)(keys[i] & 0xffffffffu);
            B_out[np] = j - i;
        }
        np++;
        i = j;
    }
    free(keys);
    return np;
}

double orc_fuse_energy(const orc_params* p, const int64_t* n, const double* S, int32_t a, int32_t b, int64_t B)
{
    double na = (double)n[a], nb = (double)n[b];
    double w = (na * nb) / (na + nb);
    double d = S[a] / na - S[b] / nb;
    return w * (d * d) - p->lambda * (double)B;
}

int64_t orc_fuse(const orc_params* p, const void* I, int32_t* L)
{
    int M = p->nlabels;
    int64_t npix = p->D * p->H * p->W;
    int64_t np = orc_fuse_pairs(p, L, NULL, NULL, NULL, 0);
    size_t cap = (size_t)(np > 0 ? np : 1);
    int32_t* a = (int32_t*)malloc(sizeof(int32_t) * cap);
    int32_t* b = (int32_t*)malloc(sizeof(int32_t) * cap);
    int64_t* B = (int64_t*)malloc(sizeof(int64_t) * cap);
    orc_fuse_pairs(p, L, a, b, B, np);
    int64_t* n = (int64_t*)malloc(sizeof(int64_t) * (size_t)M);
    double* S = (double*)malloc(sizeof(double) * (size_t)M);
    double* Q = (double*)malloc(sizeof(double) * (size_t)M);
    orc_stats(p, I, L, n, S, Q);
    fuse_pair* cand = (fuse_pair*)malloc(sizeof(fuse_pair) * cap);
    int64_t nc = 0;
    for (int64_t k = 0; k < np; k++) {
        double dE = orc_fuse_energy(p, n, S, a[k], b[k], B[k]);
        if (dE < 0.0) { cand[nc].dE = dE; cand[nc].a = a[k]; cand[nc].b = b[k]; nc++; }
    }
    qsort(cand, (size_t)nc, sizeof(fuse_pair), cmp_fuse);
    char* used = (char*)calloc((size_t)M, 1);
    int32_t* target = (int32_t*)malloc(sizeof(int32_t) * (size_t)M);
    for (int m = 0; m < M; m++) target[m] = m;
    int64_t nf = 0;
    for (int64_t k = 0; k < nc; k++) {
        if (used[cand[k].a] || used[cand[k].b]) continue;
        used[cand[k].a] = used[cand[k].b] = 1;
        target[cand[k].b] = cand[k].a;
        nf++;
    }
    if (nf)
        for (int64_t i = 0; i < npix; i++) L[i] = target[L[i]];
    free(a); free(b); free(B); free(n); free(S); free(Q); free(cand); free(used); free(target);
    return nf;
}

void orc_state_init(const orc_params* p, orc_state* st)
{
    st->mode = p->gradient;          /* 0 = Sobolev, 1 = L2, 2 = Sobolev with E = |Gamma| */
    st->converged = 0;
    st->t = 0;
    st->best_A = -1;
    st->t_best = 0;
    st->nlabels = p->nlabels;
    st->pad_ = 0;
}

/* Oscillation fallback and convergence (reading of the Eq. 6 discussion): after an iteration
 * run in mode `mode_used` that accepted `na` moves, record a new minimum of the accepted-move
 * count (strictly smaller than every earlier one), switch to L2 for good when the last new
 * minimum lies osc_window or more iterations back, and mark convergence after an L2 iteration
 * with no accepted move. */
void orc_advance_mode(const orc_params* p, orc_state* st, int32_t mode_used, int64_t na)
{
    if (st->best_A < 0 || na < st->best_A) { st->best_A = na; st->t_best = st->t; }
    if (st->mode != 1 && p->osc_window > 0 && st->t - st->t_best >= p->osc_window) st->mode = 1;
    if (mode_used == 1 && na == 0) st->converged = 1;
    st->t++;
}

int orc_iterate(const orc_params* p, const void* I, int32_t* L, orc_state* st,
                orc_status* status, int64_t cap, const orc_dump* dump)
{
    memset(status, 0, sizeof *status);
    status->mode_used = st->mode;
    if (st->converged) { status->converged = 1; st->t++; return 0; }
    orc_params q_cur = *p;
    q_cur.nlabels = st->nlabels > p->nlabels ? st->nlabels : p->nlabels;   /* labels made by splits */
    p = &q_cur;
    int M = p->nlabels;
    int64_t npix = p->D * p->H * p->W;
    int64_t* n = (int64_t*)malloc(sizeof(int64_t) * (size_t)M);
    double* S = (double*)malloc(sizeof(double) * (size_t)M);
    double* Q = (double*)malloc(sizeof(double) * (size_t)M);
    orc_stats(p, I, L, n, S, Q);
    int64_t N = orc_extract(p, L, NULL, NULL, NULL, 0);
    size_t NN = (size_t)(N > 0 ? N : 1);
    uint32_t* idx = (uint32_t*)malloc(sizeof(uint32_t) * NN);
    int32_t* l = (int32_t*)malloc(sizeof(int32_t) * NN);
    int32_t* c = (int32_t*)malloc(sizeof(int32_t) * NN);
    double* dE = (double*)malloc(sizeof(double) * NN);
    double* g = (double*)malloc(sizeof(double) * NN);
    double* A = (double*)malloc(sizeof(double) * NN);
    double* B = (double*)malloc(sizeof(double) * NN);
    double* dEs = (double*)malloc(sizeof(double) * NN);
    double* gs = (double*)malloc(sizeof(double) * NN);
    orc_extract(p, L, idx, l, c, N);
    orc_energy(p, I, L, n, S, N, idx, l, c, dE, dEs);
    if (st->mode == 0 || st->mode == 2) {
        if (st->mode == 0) {
            orc_sobolev(p, N, idx, l, c, dE, 0, g, A, B, NULL, NULL, gs);
        } else {
            /* length scale of the inner product set to the contour length (Length scale
             * section): E = |Gamma|, support |d| < E/2, every particle pair considered */
            orc_params q = *p;
            q.cutoff = 0.5 * (double)orc_perimeter(p, L);
            orc_sobolev(&q, N, idx, l, c, dE, 1, g, A, B, NULL, NULL, gs);
        }
        for (int64_t k = 0; k < N; k++)
            if (A[k] != 0.0 && B[k] != 0.0 && ((A[k] > 0.0) == (B[k] > 0.0))) status->n_osc++;
    } else {
        for (int64_t k = 0; k < N; k++) { g[k] = dE[k]; gs[k] = dEs[k]; }
    }
    uint32_t* acc_idx = (uint32_t*)malloc(sizeof(uint32_t) * NN);
    int32_t* acc_c = (int32_t*)malloc(sizeof(int32_t) * NN);
    int64_t ncand = 0;
    int64_t na = orc_select(p, L, N, idx, l, c, g, acc_idx, acc_c, &ncand);
    /* moves admitted by the split rule (judged on the labels before the moves) */
    int64_t n_split = 0;
    if (p->topology & 2)
        for (int64_t t = 0; t < na; t++) {
            int32_t l0 = L[acc_idx[t]];
            if (l0 != 0 && !simple_for_label(p, L, acc_idx[t], l0) && foreground_number(p, L, acc_idx[t], l0) >= 2)
                n_split++;
        }
    for (int64_t t = 0; t < na; t++) L[acc_idx[t]] = acc_c[t];
    if (n_split > 0) st->nlabels = orc_relabel(p, L, p->nlabels);
    if ((p->topology & 4) && p->model == 0) {
        orc_params q = *p;
        q.nlabels = st->nlabels > p->nlabels ? st->nlabels : p->nlabels;
        orc_fuse(&q, I, L);
    }
    (void)npix;
    status->n_particles = N;
    status->n_candidates = ncand;
    status->n_accepted = na;
    if (dump) {
        for (int64_t k = 0; k < N && k < cap; k++) {
            if (dump->idx) dump->idx[k] = idx[k];
            if (dump->l) dump->l[k] = l[k];
            if (dump->c) dump->c[k] = c[k];
            if (dump->dE) dump->dE[k] = dE[k];
            if (dump->g) dump->g[k] = g[k];
            if (dump->dE_terms) dump->dE_terms[k] = dEs[k];
            if (dump->g_terms) dump->g_terms[k] = gs[k];
        }
    }
    orc_advance_mode(p, st, status->mode_used, na);
    status->converged = st->converged;
    free(n); free(S); free(Q); free(idx); free(l); free(c); free(dE); free(g); free(A); free(B);
    free(dEs); free(gs);
    free(acc_idx); free(acc_c);
    return 0;
}
