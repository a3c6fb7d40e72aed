/* seg.h - C-ABI of libseg: particle region-competition segmentation with
 * particle-approximated Sobolev gradients on one CUDA GPU (sm_103a).
 *
 * Method: Sbalzarini, Schneider & Cardinale, "Particle methods enable fast and
 * simple approximation of Sobolev gradients in image segmentation" (arXiv:1403.0240).
 * One iteration (seg_step) does, entirely on the device:
 *   1. particle extraction: every (pixel x, candidate label c) with c != L(x) the
 *      label of a connectivity neighbour of x (Fig. 1; "Discrete particle
 *      approximation"), binned into a cell list of edge >= E/2 ("cell lists");
 *   2. the per-particle energy difference dE of moving x to c (Methods, Eq. 11):
 *      piecewise-constant or piecewise-smooth data term plus lambda times the
 *      change of the number of unlike neighbour pairs (length prior, Eq. 10);
 *   3. the Sobolev gradient of Eq. 6 with the kernel of Eq. 5 (eps = 1/24,
 *      E = 2 * cutoff), or dE itself in L2 mode;
 *   4. ranking and moves: per pixel the smallest gradient is a candidate if it is
 *      negative; candidates whose move keeps every foreground region's topology
 *      (simple points, 4/8 in 2D, 6/26 in 3D) are accepted greedily in ascending
 *      (gradient, pixel) order, none within Chebyshev distance 1 of another
 *      ("The Region Competition (RC) algorithm": ranking makes the result
 *      independent of particle order);
 *   5. label update and exact region statistics (count, sum I, sum I^2; the
 *      region mean is the piecewise-constant intensity, Methods);
 *   6. the oscillation fallback to L2 gradients (Eq. 6 discussion).
 * Gradients are computed in FP32 with a rigorous error bound; any ranking or sign
 * decision the bound cannot certify is recomputed in FP64 in ascending particle
 * key order, so labels are identical to an FP64 evaluation of the same rules.
 *
 * Conventions: every call returns SEG_OK (0) or a negative SEG_E* code; nothing
 * aborts the process. Pointers marked "host or device" may point to host memory
 * (pageable or pinned) or to device memory of the context's device; the library
 * tells them apart with cudaPointerGetAttributes. The caller keeps ownership of
 * everything it passes; the library copies inputs at seg_init and owns its
 * device state until seg_destroy. A context is not thread-safe: use one context
 * per host thread, or serialise calls. All work is ordered on the CUDA stream
 * given at seg_init.
 */
#ifndef SEG_H
#define SEG_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEG_OK        0
#define SEG_EINVAL   -1   /* bad parameter, shape, label image or pointer */
#define SEG_ENOMEM   -2   /* device memory (or the batch budget) exhausted */
#define SEG_ECUDA    -3   /* a CUDA runtime call failed; see seg_last_cuda_error */
#define SEG_ETIMEOUT -4   /* a bounded device-side wait gave up; the context is poisoned */
#define SEG_ESTATE   -5   /* call not valid in the object's current state */

enum { SEG_F32 = 0, SEG_U16 = 1 };                 /* image element type */
/* region models: piecewise constant (Gaussian noise, region means); piecewise smooth (local
 * means over a ball of radius R, Gaussian noise); piecewise smooth with Poisson noise: the
 * data term of a pixel is mu - I ln mu for its local mean mu (the log(I!) term dropped), the
 * means floored at 2^-20 max(1, max I); intensities must be >= 0 */
enum { SEG_PC = 0, SEG_PS = 1, SEG_PS_POISSON = 2, SEG_PC_DECONV = 3 };
/* SEG_PC_DECONV, the deconvolving piecewise-constant model (Methods, Eq. 8: the expected image
 * is J = s_theta(Gamma) * K, K the microscope's point-spread function): s_theta(x) = theta of
 * the region of x, theta the region means; K = k(x) k(y) [k(z)], a symmetric 1D profile k
 * given by seg_set_psf, zero outside the image. Data term sum_x (I(x) - J(x))^2; a move of x
 * from l to c is evaluated with theta held: dE = d^2 |K_x|^2 - 2 d G(x) + lambda dP with
 * d = theta_c - theta_l, G = K * (I - J) and |K_x|^2 = sum over in-image y of K(y - x)^2.
 * J and G are recomputed every iteration in FP64 by separable passes along x, then y, then z,
 * each output the fused multiply-add chain sum_{u=-r..r} k(u) f(. + u) in ascending u. */
#define SEG_PSF_MAX_RADIUS 512
/* gradient type at start. SEG_SOBOLEV_GLOBAL: Eq. 6 with the length scale of the inner
 * product set to the contour length, E = |Gamma| (Length scale section), |Gamma| read as the
 * number of connectivity-adjacent pixel pairs with different labels (the length prior's
 * count) and updated every iteration; the support |d| < E/2 then covers (nearly) every
 * particle pair, so the interaction is all-pairs, O(N^2) per iteration (the paper leaves this
 * variant to future work as too costly on its CPU). The cutoff parameter only sizes the cell
 * list in this mode. */
enum { SEG_SOBOLEV = 0, SEG_L2 = 1, SEG_SOBOLEV_GLOBAL = 2 };
/* topological control, bits of seg_params.topology (Particle-based image segmentation: foreground
 * regions stay connected sets; the paper's experiments disallow region fusions):
 * SEG_TOPO_VANISH - a region may vanish: the removal of its last pixel is admissible;
 * SEG_TOPO_SPLIT  - a region may split: a removal whose foreground topological number is >= 2
 *                   (it locally disconnects the region) is admissible, so the region splits or
 *                   one of its holes opens; after the moves of the iteration every foreground
 *                   label's connectivity components but the one holding its smallest pixel
 *                   index get new labels, numbered upward from the label count in ascending order
 *                   of the components' smallest pixel indices (seg_info reports the count).
 * SEG_TOPO_FUSE   - touching regions may fuse (SEG_PC with SEG_STATS_EXACT only): after the
 *                   moves (and the relabelling of split pieces), two touching foreground
 *                   labels a < b fuse when dE = w (d d) - lambda B_ab < 0, w = (n_a n_b) /
 *                   (n_a + n_b), d = S_a / n_a - S_b / n_b (statistics after the moves, FP64 as
 *                   written), B_ab their connectivity-adjacent pixel pairs: the exact change of
 *                   the squared deviations about the joint mean minus the shared contour.
 *                   Pairs are taken in ascending (dE, a, b), each label at most once per
 *                   iteration; b's pixels take label a and b stays empty. More touching pairs
 *                   than the pair table holds (max(4096, 16 M) rounded up to a power of two,
 *                   at most 2^22) end the iteration with SEG_ENOMEM. */
enum { SEG_TOPO_STRICT = 0, SEG_TOPO_VANISH = 1, SEG_TOPO_SPLIT = 2, SEG_TOPO_FUSE = 4 };
/* regulariser of the energy difference (seg_params.regulariser):
 * SEG_REG_LENGTH    - lambda * dP, dP the change of the number of connectivity-adjacent pixel
 *                     pairs with different labels (the length prior of Eq. 10);
 * SEG_REG_CURVATURE - curvature regularisation from the pixel counts of a ball (RC's sphere
 *                     estimate; integral invariants of Pottmann et al. 2007): moving x from l to
 *                     c adds w (A_l(x) - A_c(x)), A_m(x) the pixels of label m within distance
 *                     curv_radius = rho of x (x counted in l, pixels outside the image in
 *                     neither), w = lambda * (3.0 / (2.0 * (rho*rho*rho))) in 2D and
 *                     lambda * (4.0 / (pi * (rho*rho*rho*rho))) in 3D, evaluated in FP64 as
 *                     written: the first variation of |Gamma| with each region's curvature
 *                     taken from its share of the ball. */
enum { SEG_REG_LENGTH = 0, SEG_REG_CURVATURE = 1 };
/* region sums of I and I^2 (precision study; counts are exact int64 in every mode):
 * SEG_STATS_EXACT   - exact (int64 fixed point), rounded once to FP64: the means are the FP64
 *                     definition's bit for bit, results are reproducible (default);
 * SEG_STATS_F64     - FP64 sums (atomic adds, order not fixed);
 * SEG_STATS_KAHAN32 - compensated FP32 sums: a (sum, compensation) pair of floats per sum, each
 *                     addition a Neumaier step applied atomically (order not fixed).
 * In the two inexact modes the means carry the sums' rounding error: decisions are certified
 * and recomputed against FP64 evaluations that use those means, and results may vary from run
 * to run. seg_stats reports the sums each mode keeps. */
enum { SEG_STATS_EXACT = 0, SEG_STATS_F64 = 1, SEG_STATS_KAHAN32 = 2 };

typedef struct seg_ctx seg_ctx;
typedef struct seg_batch seg_batch;

typedef struct {
    int32_t ndim;          /* 2 | 3 */
    int32_t dtype;         /* SEG_F32 | SEG_U16 */
    int64_t shape[3];      /* {D, H, W}; D = 1 in 2D; row-major, x fastest; each >= 1, D*H*W < 2^31 */
    int32_t model;         /* SEG_PC | SEG_PS | SEG_PS_POISSON | SEG_PC_DECONV */
    int32_t connectivity;  /* foreground: 4 (2D) | 6 (3D); background uses 8 | 26 */
    double  lambda;        /* length weight (Eq. 10), >= 0 */
    double  cutoff;        /* interaction cutoff E/2 in pixels, > 0; E = 2 * cutoff, eps = 1/24 */
    double  ps_radius;     /* local-mean radius R for SEG_PS and SEG_PS_POISSON, >= 1 */
    int32_t gradient;      /* SEG_SOBOLEV | SEG_L2 | SEG_SOBOLEV_GLOBAL */
    int32_t osc_window;    /* switch to L2 once the accepted-move count has not reached a new
                              minimum for this many iterations; 0 = never switch */
    int32_t stats_mode;    /* SEG_STATS_EXACT | SEG_STATS_F64 | SEG_STATS_KAHAN32 */
    int32_t validate;      /* nonzero: check on the host that every foreground label of labels0
                              is one connected component (else SEG_EINVAL) */
    int32_t cell_edge;     /* cell-list edge in pixels, >= ceil(cutoff); 0 = ceil(cutoff) */
    int32_t tile[3];       /* tile shape in pixels {z, y, x}, each 0 (default) or 1..1024; a tile
                              is floor(tile / cell_edge) cells (at least one) per axis; z must be
                              0 or 1 in 2D. Default 8 x 32 x 32 / cell (3D), 32 x 64 / cell (2D) */
    int32_t topology;      /* SEG_TOPO_STRICT (0: every move keeps each foreground region one
                              connected component with its holes) or an OR of SEG_TOPO_VANISH,
                              SEG_TOPO_SPLIT and SEG_TOPO_FUSE */
    int32_t max_labels;    /* with SEG_TOPO_SPLIT: label capacity (labels 0..max_labels-1), >= the
                              initial count; 0 = max(2 M, M + 256) for M initial labels. A split
                              beyond it ends the iteration with SEG_ENOMEM. Ignored otherwise */
    int32_t regulariser;   /* SEG_REG_LENGTH (0): lambda * change of the unlike neighbour pairs;
                              SEG_REG_CURVATURE (1): curvature from ball counts, see below */
    int32_t reserved;      /* must be zero */
    double  curv_radius;   /* SEG_REG_CURVATURE: ball radius rho, 1 <= rho <= 16; ignored otherwise */
} seg_params;

typedef struct {
    int64_t iteration;     /* index of the iteration this status describes (0-based) */
    int64_t n_particles;
    int64_t n_candidates;  /* pixels whose best particle is negative and topology-admissible */
    int64_t n_accepted;    /* moves executed */
    int64_t n_osc;         /* particles whose two Eq. 6 terms are non-zero with equal sign (FP32) */
    int64_t n_fixup;       /* particles whose gradient was recomputed in FP64 */
    int32_t mode_used;     /* SEG_SOBOLEV | SEG_L2 | SEG_SOBOLEV_GLOBAL */
    int32_t converged;     /* an L2 iteration accepted no move; later iterations do nothing */
    int32_t mis_rounds;    /* rounds of the parallel ranked selection (many candidates: the most sweeps of one block) */
    int32_t error;         /* 0, or a SEG_E* code raised on the device; SEG_ENOMEM: the
                              particle buffers overflowed and the iteration was not run
                              (the next seg_step regrows them and runs it) */
    int64_t particles_total; /* particles summed over all iterations run so far */
} seg_status;

typedef struct {
    int64_t t;             /* iterations done */
    int64_t best_A;        /* smallest accepted-move count so far (-1 before the first iteration) */
    int64_t t_best;        /* iteration at which best_A was first reached */
    int32_t mode;          /* SEG_SOBOLEV | SEG_L2 | SEG_SOBOLEV_GLOBAL */
    int32_t converged;
} seg_state;

/* Particle arrays of the most recent iteration, in the library's internal order
 * (cell-major; sort by (idx, c) to get key order). Each pointer may be NULL (not
 * copied), host or device. */
typedef struct {
    uint32_t* idx;         /* linear pixel index (z*H + y)*W + x */
    int32_t*  l;           /* current label of the pixel */
    int32_t*  c;           /* candidate label */
    float*    dE;          /* L2 energy difference (FP32) */
    float*    eE;          /* bound on |dE - dE_fp64| */
    float*    g;           /* gradient used for ranking: Eq. 6 in Sobolev mode, dE in L2 mode */
    float*    eg;          /* bound on |g - g_fp64| */
    double*   key;         /* ranking key: the FP64 value where recomputed, else g */
    uint8_t*  flags;       /* bit 0 recomputed in FP64, bit 1 pixel candidate, bit 2 accepted */
} seg_particle_buffers;

/* Bytes of device memory seg_init will allocate for these parameters (particle
 * capacity at its initial size). Returns SEG_EINVAL for invalid parameters. */
int seg_estimate_bytes(const seg_params* p, int32_t nlabels, size_t* bytes);

/* Autotuning (batched and served workloads): the cell-list edge and the tile shape change only
 * the speed, never a label, statistic or particle set. seg_autotune times candidates on the
 * given job: cell edge in {c, 2c} (c = p->cell_edge, or ceil(cutoff) when 0) times tile shapes
 * {16x16, 32x32, 32x64, 64x64, 64x128} (2D, y x x) or {8x8x8, 8x8x32, 16x16x16, 8x16x32,
 * 16x16x32} (3D, z x y x x); a candidate whose tiles come out the same in cells as an earlier
 * one is skipped. Each candidate is a fresh context (seg_init on image and labels0, host or
 * device pointers) stepped 2 untimed and then `iters` timed iterations (CUDA events on
 * cuda_stream; no L2 flush); its mean time per iteration is reported. *best receives p with
 * cell_edge and tile set to the fastest candidate. entries (may be NULL) receive up to
 * max_entries candidates in the order tried, *n_entries (may be NULL) their number.
 * Returns SEG_OK when at least one candidate ran, else the first candidate's error (for
 * SEG_PC_DECONV, which needs its PSF before a step, every candidate fails with SEG_ESTATE: tune
 * such jobs with the piecewise-constant model on the same image: the settings act on the same
 * extraction and interaction kernels). */
typedef struct {
    int32_t cell_edge;     /* cell-list edge in pixels */
    int32_t tile[3];       /* tile shape in pixels {z, y, x} */
    float   ms_per_iter;   /* mean time of one iteration; -1 when the candidate failed */
    int32_t status;        /* SEG_OK, or the error seg_init / seg_step returned */
} seg_tune_entry;

int seg_autotune(const seg_params* p, const void* image, const int32_t* labels0, int32_t iters,
                 void* cuda_stream, seg_params* best, seg_tune_entry* entries, int32_t max_entries,
                 int32_t* n_entries);

/* Create a context: validates p, copies image (dtype elements, D*H*W, host or
 * device) and labels0 (int32 >= 0, host or device; 0 = background), computes the
 * exact region statistics. cuda_stream is a cudaStream_t (NULL = the legacy default
 * stream) on the current device. Errors: SEG_EINVAL (parameters, shape, negative
 * labels, non-finite image values, a disconnected foreground label when
 * p->validate), SEG_ENOMEM, SEG_ECUDA. On error *out is NULL. */
int seg_init(const seg_params* p, const void* image, const int32_t* labels0,
             void* cuda_stream, seg_ctx** out);

/* Deconvolving model (SEG_PC_DECONV, Eq. 8): set the PSF profile k(-radius..radius), 2 radius + 1
 * host doubles, read during the call; finite and symmetric (k(u) == k(-u) exactly);
 * 0 <= radius <= SEG_PSF_MAX_RADIUS. The PSF is K = k(x) k(y) [k(z)] on every axis. Required
 * before the first step of such a context (a step without it returns SEG_ESTATE); may be
 * called again between steps, the next iteration then uses the new PSF. Synchronises the
 * context's stream. Errors: SEG_EINVAL (arguments), SEG_ESTATE (another model). */
int seg_set_psf(seg_ctx* c, const double* k, int32_t radius);

/* Run iters iterations (iters >= 0) on the context's stream, replaying one
 * captured CUDA graph per iteration, and wait for them. If out is not NULL it
 * receives the status of the last iteration. Returns the device error code if
 * one was raised (SEG_ETIMEOUT), SEG_ECUDA on a runtime failure. */
int seg_step(seg_ctx* c, int32_t iters, seg_status* out);

/* Enqueue iters iterations on the context's stream and return without waiting
 * (graph launches only; no host synchronisation, no buffer regrowth). */
int seg_step_async(seg_ctx* c, int32_t iters);

/* Wait for the context's stream and return the status of the last iteration run. */
int seg_poll(seg_ctx* c, seg_status* out);

/* Stage timing: when on, the captured iteration graph also records CUDA events
 * between its stages (psf, extract, sobolev, select, lists, fixup, rounds, moves, finish;
 * psf is the deconvolving model's field passes, empty for the other models; sobolev includes
 * the candidate selection, and select is the E = |Gamma| mode's own selection, empty
 * otherwise; lists includes the order certificates of neighbouring candidates, fixup the FP64
 * recompute of the keys they did not certify); seg_stage_times waits for the stream and writes
 * the milliseconds
 * each stage took in the most recent iteration (n >= 9), returning SEG_ESTATE when timing
 * is off. */
int seg_profile(seg_ctx* c, int32_t on);
int seg_stage_times(seg_ctx* c, float* ms, int32_t n);

/* Copy the current label image (D*H*W int32) to out (host or device); n_out is
 * the element capacity of out (SEG_EINVAL if too small). Synchronises the stream. */
int seg_labels(seg_ctx* c, int32_t* out, size_t n_out);

/* Copy the particle arrays of the most recent iteration (up to cap entries) and
 * store their count in *n. Synchronises the stream. */
int seg_particles(seg_ctx* c, const seg_particle_buffers* out, int64_t cap, int64_t* n);

/* Region statistics for labels 0..max_labels-1 (host arrays, each may be NULL):
 * count, sum of I and sum of I^2 over the region, exact and rounded once (the sums of
 * squares are rounded by this call). Call it between steps: it synchronises the context's
 * stream, not a batch's step in flight. */
int seg_stats(seg_ctx* c, int64_t* n, double* S, double* Q, int32_t max_labels);

/* Optimiser state for checkpointing; seg_set_state restores it after a seg_init
 * from the saved labels, so that the next iterations repeat bit for bit. */
int seg_get_state(seg_ctx* c, seg_state* out);
int seg_set_state(seg_ctx* c, const seg_state* in);

/* Number of labels M (max label of labels0 + 1) and the image shape. */
int seg_info(seg_ctx* c, int32_t* nlabels, int64_t shape[3]);

void seg_destroy(seg_ctx* c);

/* Batching: contexts on the same device stepped together, one launch per stage
 * for all of them (continuous batching adds and removes contexts between steps).
 * The batch does not own the contexts; a context belongs to at most one batch. */
int seg_batch_create(void* cuda_stream, seg_batch** out);
int seg_batch_add(seg_batch* b, seg_ctx* c);
int seg_batch_remove(seg_batch* b, seg_ctx* c);
int seg_batch_size(seg_batch* b);
/* Run iters iterations of every context in the batch; statuses (may be NULL)
 * receives one seg_status per context in the order they were added. */
int seg_batch_step(seg_batch* b, int32_t iters, seg_status* statuses, int32_t n_statuses);
int seg_batch_step_async(seg_batch* b, int32_t iters);
/* Per-stage CUDA events of the batch's iteration, as seg_profile / seg_stage_times for one
 * context (the events serialise the stage launches, so profiled steps run slower): ms
 * (n >= 9) receives the milliseconds each of the nine stages took in the batch's most recent
 * iteration, over all members together. */
int seg_batch_profile(seg_batch* b, int32_t on);
int seg_batch_stage_times(seg_batch* b, float* ms, int32_t n);
int seg_batch_poll(seg_batch* b, seg_status* statuses, int32_t n_statuses);
void seg_batch_destroy(seg_batch* b);

/* Exact region statistics of a label image, allocating no device memory.
 * The paper has no counterpart: this is for callers that cannot call cudaMalloc, such as
 * code that manages device memory through a pool of its own (an unplanned cudaMalloc would
 * bypass the pool's accounting and can fragment or exhaust it) or code that must not risk
 * the implicit device synchronisation of cudaMalloc/cudaFree. It computes what seg_init
 * computes and seg_stats returns: per label m < nlabels the pixel count n[m], and the sums
 * S[m] of I and Q[m] of I^2 over the region, each exact and rounded once to FP64.
 * image (dtype elements), labels (int32 in 0..nlabels-1), n (int64), S and Q (double) are
 * caller-owned device buffers of npix and nlabels elements; host pointers give SEG_EINVAL.
 * Limits: 1 <= nlabels <= 1024 and npix < 2^31, else SEG_EINVAL; a label outside
 * 0..nlabels-1 gives SEG_EINVAL before anything is summed. Non-finite float values give
 * meaningless sums but stay in bounds.
 * The working accumulators live in one fixed device array of about 6.6 MB that every GPU
 * loading libseg holds until the process exits. The first call on a device looks up that
 * array's device address (once per device), so make it before any stream capture. Under CUDA's
 * lazy module loading that first look-up may also load libseg's device code on that device,
 * which reserves the array and can synchronise the device: a caller with a strict rule against
 * allocation or synchronisation should make one warm-up call at start-up. All calls
 * share the array, so calls that overlap on the GPU (other streams, other host threads)
 * race and give wrong results. Work is ordered on cuda_stream (a cudaStream_t, NULL = the
 * legacy default stream); the call returns after it has finished. */
int seg_region_stats_noalloc(int32_t dtype, int64_t npix, const void* image, const int32_t* labels,
                             int32_t nlabels, int64_t* n, double* S, double* Q, void* cuda_stream);

/* Test hook: the device's simple-point test on n neighbourhood bitmasks (host arrays).
 * Bit k of masks[i] is neighbour k of the 3x3 (2D, 8 bits) or 3x3x3 (3D, 26 bits) window
 * in row-major order with the centre left out; out[i] = 1 if the centre is a simple
 * point (4/8 in 2D, 6/26 in 3D). */
int seg_debug_simple(int32_t ndim, const uint32_t* masks, int32_t n, uint8_t* out);

/* Test-only fault injection, for checking that bounded device waits report instead of
 * hanging. SEG_INJECT_WITHHELD_COPY: from the next iteration on, extraction's first tile
 * arms its barrier for the label copy but issues no copy (when labels arrive by tensor copies,
 * i.e. rows of a multiple of 16 bytes), so its bounded wait runs out (about two seconds), and so
 * do the waits of the tiles after it for its particle count; the iteration ends with
 * SEG_ETIMEOUT and the context is then poisoned (destroy it).
 * SEG_INJECT_NONE clears the injection. No GPU fault is raised. */
enum { SEG_INJECT_NONE = 0, SEG_INJECT_WITHHELD_COPY = 1 };
int seg_debug_inject(seg_ctx* c, int32_t what);

/* Kernels libseg has launched in this process so far (all devices and threads); each replay
 * of an iteration graph counts every kernel of the graph. For measuring how many kernels a
 * piece of work takes: read it before and after. */
int seg_kernel_launches(uint64_t* out);

const char* seg_strerror(int code);
/* Text of the last CUDA error this thread saw inside libseg ("" if none). */
const char* seg_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif
