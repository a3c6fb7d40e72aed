/* rc_oracle.h - CPU oracle for particle region competition with Sobolev gradients.
 *
 * TEST INFRASTRUCTURE ONLY. This plain, slow, single-threaded FP64 implementation
 * of one iteration of the method of Sbalzarini, Schneider & Cardinale, "Particle
 * methods enable fast and simple approximation of Sobolev gradients in image
 * segmentation" (arXiv:1403.0240) exists to check the CUDA path. Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may load it. It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Parity status of each function (what pins it, in tests/test_oracle_*.py):
 *   orc_kernel_eq5      - Eq. 5; pinned by the closed form at eps = 1/24, the
 *                         Figure 2 axis ticks, the vanishing at r = +-E/2, unit mass.
 *   orc_extract         - particles on either side of the contour (Fig. 1); pinned
 *                         by the 64x64 square count (252 inner + 256 outer) and a
 *                         numpy brute-force neighbour scan.
 *   orc_stats           - exact region sums rounded once; pinned by math.fsum,
 *                         fractions.Fraction and the partition invariants.
 *   orc_energy (PC)     - exact single-flip SSE change; pinned by a brute-force
 *                         recompute of the total SSE before and after the flip.
 *   orc_energy (PS)     - local-mean difference; pinned by scipy.ndimage
 *                         convolutions and by the R -> infinity limit.
 *   orc_energy (Poisson)- f(v, mu_c) - f(v, mu_l), f(v, mu) = mu - v ln mu over the same
 *                         local means; pinned by convolutions and numpy logarithms.
 *   orc_log             - pinned against the C library logarithm within 4 ulp.
 *   orc_energy (deconv) - -2 d G(x) + d^2 |K_x|^2 with d = theta_c - theta_l, G = K * (I - K * s);
 *                         pinned by a brute-force recompute of sum (I - K * s)^2 before and
 *                         after the flip (numpy/scipy, theta held), and by K = delta reducing
 *                         to the fixed-mean single-pixel SSE change.
 *   orc_psf_correlate   - pinned by scipy.ndimage.correlate with the outer-product kernel
 *                         and by the impulse response (exactly the outer product).
 *   orc_energy (length) - pinned by a brute-force recount of the perimeter.
 *   orc_sobolev         - Eq. 6 with a cell list; pinned by all-pairs brute force,
 *                         the degenerate cutoff, and a hand-computed straight line.
 *   orc_simple_2d/3d    - topological numbers; pinned by Yokoi's formula and global
 *                         component counts (2D), and by contractibility of the
 *                         centre's link in the cubical complex (3D).
 *   orc_admissible      - with topology 1, the removal of a region's last pixel is admissible;
 *                         pinned by global pixel counts on random connected label images and
 *                         by a one-pixel region that vanishes. With topology 2 a removal whose
 *                         foreground topological number is >= 2 is admissible; pinned by a
 *                         dumbbell whose neck is removed, and by global component counts.
 *   relabelling (topology 2) - pinned by scipy.ndimage.label components and the numbering rule.
 *   orc_fuse_pairs      - touching foreground pairs and their shared pixel pairs B_ab; pinned
 *                         by a perimeter recount (P before minus P after renaming b to a).
 *   orc_fuse_energy     - n_a n_b/(n_a + n_b) (mu_a - mu_b)^2 - lambda B_ab; pinned by brute-force
 *                         total energies (squared deviations plus lambda P) before and after.
 *   orc_fuse            - greedy matching of the negative pairs; pinned by a greedy pass over
 *                         brute-force energies (a matching, maximal, the energy falls).
 *   orc_ball_balance,   - curvature regulariser w (A_l - A_c); pinned by the exact count on a
 *   orc_curvature_weight  straight edge (the ball's central row or plane), the curvature of
 *                         digital disks (1/R) and spheres (2/R) from the inner and outer
 *                         particles, and a brute-force count with image borders.
 *   orc_select          - ranked greedy selection; pinned by an independent
 *                         local-minimum-rounds evaluation and permutation tests.
 *   orc_perimeter       - |Gamma| as the length prior counts it; pinned by square and
 *                         cube perimeters and a numpy recount.
 *   orc_advance_mode    - pinned by hand-worked accepted-move sequences with their switch and
 *                         convergence iterations (tests/golden/osc_switch.txt).
 *   term sums           - the tolerance scale of dE and g (Sum |terms|); pinned by term-by-term
 *                         numpy recomputes from the region statistics and the Eq. 6 sets.
 *   orc_iterate         - composition of the above; pinned by the partition and
 *                         connectivity invariants after every iteration. With E = |Gamma|
 *                         (gradient 2) the Sobolev step is the all-pairs Eq. 6 at E = the
 *                         perimeter; pinned by a numpy evaluation of Eq. 6 over all pairs.
 */
#ifndef RC_ORACLE_H
#define RC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t ndim;        /* 2 | 3 */
    int32_t dtype;       /* 0 = float32 image, 1 = uint16 image */
    int64_t D, H, W;     /* D = 1 in 2D; row-major, x fastest */
    int32_t model;       /* 0 = piecewise constant, 1 = piecewise smooth (Gaussian noise),
                            2 = piecewise smooth with Poisson noise, 3 = deconvolving piecewise
                            constant (J = s_theta * K, Eq. 8) */
    int32_t conn;        /* foreground connectivity: 4 (2D) | 6 (3D) */
    double lambda;       /* length weight (Eq. 10) */
    double cutoff;       /* interaction cutoff E/2 in pixels */
    double ps_radius;    /* local-mean radius R (piecewise smooth) */
    int32_t gradient;    /* 0 = Sobolev (Eq. 6), 1 = L2, 2 = Sobolev with E = |Gamma| (all pairs) */
    int32_t osc_window;  /* iterations without a new minimum of accepted moves before switching to L2; 0 = never */
    int32_t nlabels;     /* M: labels are 0..M-1 */
    int32_t pad_;
    double mu_floor;     /* Poisson model: local means below this are taken as this */
    int32_t psf_r;       /* deconvolving model: PSF profile radius r (psf has 2r + 1 taps) */
    int32_t topology;    /* topological control, bits: 0 = every move keeps each region's topology;
                            1 = a region may vanish (its last pixel may leave it); 2 = a region may
                            split (a removal that locally disconnects it is admissible; after the
                            moves of an iteration with such a move, every foreground label's
                            components but the one holding its smallest pixel index get new
                            labels); 4 = touching regions may fuse (piecewise-constant model:
                            after the moves, pairs whose fusion lowers the energy, see orc_fuse) */
    const double* psf;   /* deconvolving model: symmetric 1D PSF profile k(-r..r), the same on
                            every axis (K(x) = prod_axes k(x_a)) */
    int32_t regulariser; /* 0 = length prior lambda * (change of unlike neighbour pairs);
                            1 = curvature from ball counts, weight from lambda (orc_curvature_weight) */
    int32_t pad2_;
    double curv_radius;  /* regulariser 1: ball radius rho >= 1 */
} orc_params;

typedef struct {
    int32_t mode;        /* 0 = Sobolev, 1 = L2 */
    int32_t converged;
    int64_t t;           /* iterations done */
    int64_t best_A;      /* smallest accepted-move count so far, -1 before the first iteration */
    int64_t t_best;      /* first iteration at which best_A was reached */
    int32_t nlabels;     /* labels in use: p->nlabels, grown by splits */
    int32_t pad_;
} orc_state;

typedef struct {
    int64_t n_particles;
    int64_t n_candidates;
    int64_t n_accepted;
    int64_t n_osc;       /* particles whose two Eq. 6 terms are non-zero with equal sign */
    int32_t mode_used;
    int32_t converged;
} orc_status;

double  orc_kernel_eq5(double r, double E, double eps);

/* natural logarithm of x > 0 by the atanh series after reduction to [sqrt(1/2), sqrt(2)):
 * ln x = e ln 2 + 2 (y + y^3/3 + ... + y^23/23), y = (m - 1)/(m + 1); every operation an IEEE
 * double operation in a fixed order */
double  orc_log(double x);

/* Curvature regulariser: A_l(x) - A_c(x), the pixels of label l minus those of label c in the
 * ball |y - x|^2 <= rho^2 around x (x counts in its own label; pixels outside the image in
 * neither), and the weight w with which it enters the energy difference. */
int64_t orc_ball_balance(const orc_params* p, const int32_t* L, uint32_t xi, int32_t l, int32_t c);
double  orc_curvature_weight(const orc_params* p);

int64_t orc_extract(const orc_params* p, const int32_t* L,
                    uint32_t* idx, int32_t* l, int32_t* c, int64_t cap);

double  orc_exact_sum_f32(const float* v, int64_t n, int squares);

/* separable correlation with the PSF, zero outside the image: along x, then y, then z, each
 * output sum_{u=-r..r} k(u) f(. + u) in ascending u, every term added by one fma */
void    orc_psf_correlate(const orc_params* p, const double* f, double* out);

/* deconvolving model fields for the current labels: J = K * s_theta (s_theta(x) = theta_L(x),
 * theta_i = S_i / n_i), R = I - J, G = K * R; J and R may be NULL */
void    orc_deconv_fields(const orc_params* p, const void* I, const int32_t* L,
                          const int64_t* n, const double* S, double* J, double* R, double* G);

/* sum over in-image x of K(x - p)^2, factorised per axis: nrm_a(t) = sum_u k(u)^2 over the
 * u with t + u inside (ascending u, fma); returns the product over the axes */
double  orc_psf_norm2(const orc_params* p, int64_t z, int64_t y, int64_t x);

void    orc_stats(const orc_params* p, const void* I, const int32_t* L,
                  int64_t* n, double* S, double* Q);

/* scale (may be NULL): the sum of the magnitudes of the terms each dE adds up, the scale of
 * the float tolerance: PC |t1| + |t2|, PS a^2 + b^2, Poisson |m_c| + |v ln m_c| + |m_l| +
 * |v ln m_l|, deconvolving |d^2 |K_x|^2| + |2 d G|; plus |w dP| of the regulariser */
void    orc_energy(const orc_params* p, const void* I, const int32_t* L,
                   const int64_t* n, const double* S, int64_t N,
                   const uint32_t* idx, const int32_t* l, const int32_t* c, double* dE, double* scale);

int64_t orc_delta_perimeter(const orc_params* p, const int32_t* L, uint32_t x, int32_t l, int32_t c);

/* |Gamma|: connectivity-adjacent pixel pairs with different labels */
int64_t orc_perimeter(const orc_params* p, const int32_t* L);

/* scale (may be NULL): the term-magnitude sum of each g, sum_Q |K dE_q| / |Q| + sum_Q' |K dE_q| / |Q'| */
void    orc_sobolev(const orc_params* p, int64_t N, const uint32_t* idx, const int32_t* l,
                    const int32_t* c, const double* dE, int all_pairs,
                    double* g, double* A, double* B, int32_t* nQ, int32_t* nQp, double* scale);

int     orc_simple_2d(const uint8_t* nb9);
int     orc_simple_3d(const uint8_t* nb27);
int     orc_admissible(const orc_params* p, const int32_t* L, uint32_t x, int32_t l, int32_t c);

/* topology 2: give every foreground label's connectivity components but the one holding its
 * smallest pixel index new labels nlabels, nlabels + 1, ... in ascending order of the components'
 * smallest pixel indices; returns the new label count */
int32_t orc_relabel(const orc_params* p, int32_t* L, int32_t nlabels);

/* Fusion: the touching foreground label pairs a < b with their number B of connectivity-adjacent
 * pixel pairs, ascending (a, b) (returns the count; writes at most cap); the energy change of
 * fusing a pair from statistics n, S; and one fusion pass over L (returns the fusions made). */
int64_t orc_fuse_pairs(const orc_params* p, const int32_t* L, int32_t* a, int32_t* b, int64_t* B, int64_t cap);
double  orc_fuse_energy(const orc_params* p, const int64_t* n, const double* S, int32_t a, int32_t b, int64_t B);
int64_t orc_fuse(const orc_params* p, const void* I, int32_t* L);

int64_t orc_select(const orc_params* p, const int32_t* L, int64_t N,
                   const uint32_t* idx, const int32_t* l, const int32_t* c, const double* g,
                   uint32_t* acc_idx, int32_t* acc_c, int64_t* n_candidates);

void    orc_state_init(const orc_params* p, orc_state* st);

/* the mode and convergence rule applied after each iteration (see rc_oracle.c) */
void    orc_advance_mode(const orc_params* p, orc_state* st, int32_t mode_used, int64_t na);

/* per-particle arrays of one iteration, in key order (each pointer may be NULL) */
typedef struct {
    uint32_t* idx;
    int32_t* l;
    int32_t* c;
    double* dE;
    double* g;
    double* dE_terms;    /* term-magnitude sums (orc_energy's scale) */
    double* g_terms;     /* term-magnitude sums (orc_sobolev's scale; dE_terms in L2 mode) */
} orc_dump;

int     orc_iterate(const orc_params* p, const void* I, int32_t* L, orc_state* st,
                    orc_status* status, int64_t cap, const orc_dump* dump);

#ifdef __cplusplus
}
#endif
#endif
