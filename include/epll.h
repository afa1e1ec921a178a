/*
 * epll.h -- C ABI of libepll, a CUDA (sm_103a) implementation of the patch
 * step of EPLL / fast-EPLL half-quadratic-splitting image restoration
 * (Parameswaran, Deledalle, Denis & Nguyen, "Accelerating GMM-based patch
 * priors for image restoration: three ingredients for a 100x speed-up").
 *
 * Equation numbers follow their order of appearance in the paper: Eq. 1
 * EPLL objective, Eq. 2 GMM prior, Eqs. 3-5 half-quadratic splitting,
 * Algorithm 1 (patch extraction, Gaussian selection, patch estimation, patch
 * reprojection, image estimation), Eq. 6 closed-form image update, Eqs. 7-10
 * eigenspace form, Eqs. 11-16 flat-tail form, Eq. 20 jittered sampling.
 *
 * Conventions for every entry point:
 *  - images are H x W row-major float32, grey levels in [0, 1];
 *  - "device" pointers are CUDA global memory of the current device, "host"
 *    pointers are ordinary (pageable or pinned) host memory;
 *  - the caller owns every image buffer; the library owns the model handle
 *    and a scratch workspace cached inside it (grown on demand, freed with
 *    the handle); a handle must not be used by two host threads at once;
 *  - `stream` is a cudaStream_t (NULL = legacy default stream); work is
 *    enqueued on it and the call returns without synchronising unless stated;
 *  - no C++ exception crosses the ABI; every call validates its arguments and
 *    returns an epll_status; epll_last_error() gives a thread-local message;
 *    asynchronous CUDA faults surface as EPLL_ECUDA at the next call that
 *    synchronises.
 */
#ifndef EPLL_H
#define EPLL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EPLL_OK = 0,
    EPLL_EINVAL = -1,       /* bad argument: the call did nothing */
    EPLL_ENOMEM = -2,       /* device allocation failed */
    EPLL_ECUDA = -3,        /* a CUDA runtime / cuFFT call failed */
    EPLL_ETIMEOUT = -4,     /* a bounded device wait gave up */
    EPLL_EUNSUPPORTED = -5  /* valid request this build cannot serve */
} epll_status;

/* flat-tail rank selection (Sec. "Speed-up via flat tail spectrum approximation") */
enum { EPLL_RANK_FIXED = 0, EPLL_RANK_RHO = 1 };
/* degradation operator A of y = A x + w (Sec. 2); CONV_DECIMATE is the
 * super-resolution operator: the periodic blur followed by keeping pixel
 * (f i, f j) of every f x f block (f = `factor`) */
enum { EPLL_DENOISE = 0, EPLL_PIXELWISE = 1, EPLL_CONV_PERIODIC = 2, EPLL_CONV_DECIMATE = 3 };
/* patch subset (Sec. "Speed-up via the restriction to a random subset of patches"):
 * ALL every pixel's patch; FRACTION ceil(f N) distinct anchors redrawn every
 * iteration; JITTER the jittered grid of Eq. 20 (spacing s); REGULAR the
 * regular grid of spacing s, anchors (s n, s m), the same at every iteration;
 * VALID the `valid` boundary: every patch that lies inside the image (no
 * periodic wrap), with Eq. 6 taken with its non-constant overlap: the image
 * update weighs each pixel's patch average by its patch count / P (for a
 * periodic blur the update then runs cg_iters conjugate-gradient iterations
 * from the patch average instead of the Fourier solve) */
enum { EPLL_SUBSET_ALL = 0, EPLL_SUBSET_FRACTION = 1, EPLL_SUBSET_JITTER = 2, EPLL_SUBSET_REGULAR = 3,
       EPLL_SUBSET_VALID = 4 };
/* arithmetic of the projection that drives the Gaussian selection:
 * FP32   SIMT FP32 dot products;
 * BF16   tcgen05 tensor cores, BF16 operands, FP32 accumulation;
 * FP16   tcgen05 tensor cores, FP16 operands, FP32 accumulation;
 * BF16X3 tcgen05 tensor cores, operands split into hi + lo BF16 parts
 *        (three products: hi*hi + lo*hi + hi*lo), FP32 accumulation;
 * FP8    tcgen05 tensor cores (kind::f8f6f4), E4M3 operands with one scale per
 *        component and one per patch, FP32 accumulation;
 * AUTO   FP16 for models of uniform rank >= 32, BF16X3 otherwise.
 * FP16 keeps each patch's four best components; a patch it cannot decide has
 * the components within its error bound of the best rescored in the BF16X3
 * form (grouped by component on the tensor cores).  BF16 and FP8 hand the
 * patches they cannot decide to a BF16X3 pass over every component.  Every
 * form rescores its remaining near-ties (and FP16 every patch with more than
 * four components in its band) in compensated FP32 (see tie_gap).  All forms
 * select the exact argmin of Eq. 14 up to that rescoring's resolution. */
enum { EPLL_FP32 = 0, EPLL_BF16 = 1, EPLL_FP16 = 2, EPLL_BF16X3 = 3, EPLL_FP8 = 4, EPLL_AUTO = 5 };
/* how the Gaussian selection finds its candidates:
 * EXHAUSTIVE every component is scored (Algorithm 1, step 2);
 * PROPOSAL   a learned network attached to the model (epll_gmm_attach_proposal)
 *            proposes m components per patch, which are scored exactly in FP32;
 *            a patch whose proposals hold too little softmax mass, or whose two
 *            best rescored proposals are within the FP32 error bound of each
 *            other, is scored exhaustively (BF16X3, then compensated FP32
 *            rescoring of its near-ties).  `precision` is ignored. */
/* TREE       the balanced search tree attached to the model
 *            (epll_gmm_attach_tree): every patch descends from the root to a
 *            leaf, taking at each level the child with the lowest score of
 *            Eq. 14 on the node's flat-tailed Gaussian (split BF16 on the
 *            tensor cores; ties to the lowest child).  An approximation of the
 *            exhaustive argmin, as in the paper.  `precision` is ignored. */
enum { EPLL_SELECT_EXHAUSTIVE = 0, EPLL_SELECT_PROPOSAL = 1, EPLL_SELECT_TREE = 2 };

typedef struct epll_gmm epll_gmm; /* opaque, library-owned */
typedef struct epll_proposal epll_proposal; /* opaque, library-owned */

/* Degradation A.  PIXELWISE: A = diag(a) (a = 0/1 mask for inpainting, a
 * smooth gain for devignetting).  CONV_PERIODIC: circular convolution with a
 * kh x kw kernel whose centre (kh/2, kw/2) maps to pixel offset (0, 0).
 * CONV_DECIMATE (super-resolution, Sec. "Complexity via eigenspace
 * implementation" and Fig. 8): the same convolution followed by decimation by
 * `factor`; the observation y is then (H/factor) x (W/factor) while x is
 * H x W. */
typedef struct {
    int kind;
    const float *a;      /* PIXELWISE: H*W gains; device for epll_restore, host for epll_restore_host */
    const float *kernel; /* CONV_PERIODIC, CONV_DECIMATE: host, kh*kw row-major, copied during the call */
    int kh, kw;          /* 1..min(H, W) each */
    int factor;          /* CONV_DECIMATE: 1..8, dividing H and W; ignored otherwise */
} epll_degradation;

typedef struct {
    int precision;      /* EPLL_FP32, EPLL_BF16, EPLL_FP16, EPLL_BF16X3, EPLL_FP8 or EPLL_AUTO */
    float tie_gap;      /* absolute part of the near-tie threshold: a patch whose top-2
                           score gap is below tie_gap + rho * |z|^2 * max_kj 1/nu_kj is
                           rescored in compensated FP32 (rho is the relative error bound of
                           the precision: 1e-5 FP32, 1.5e-3 FP16, 1e-2 BF16, 4e-5 BF16X3,
                           1e-1 FP8; AUTO that of the form it stands for);
                           < 0 selects the default 1e-3 */
    int subset;         /* EPLL_SUBSET_* */
    double subset_param; /* FRACTION: fraction f in (0, 1], ceil(f*H*W) patches; JITTER / REGULAR: grid spacing s in 1..8;
                            ignored for ALL and VALID */
    uint64_t seed;      /* sampler seed (counter-based splitmix64 draws) */
    int cg_iters;       /* conjugate-gradient iterations (>= 0): PIXELWISE initialisation, and
                           the image update of CONV_PERIODIC with the VALID boundary */
    int select;         /* EPLL_SELECT_EXHAUSTIVE, EPLL_SELECT_PROPOSAL or EPLL_SELECT_TREE */
} epll_options;

/* Fills *o with the defaults: FP32, default tie gap, all patches, seed 0, 100 CG
 * iterations, exhaustive selection. */
void epll_options_default(epll_options *o);

/*
 * Loads a zero-mean GMM patch prior (Eq. 2) given in eigen form and prepares
 * its flat-tail approximation.
 *   K            number of components, 1..4096
 *   P            patch dimension; must be 64 (8 x 8 patches)
 *   weights      host [K], > 0; renormalised to sum 1
 *   eigvecs      host [K][P][P] row-major: eigvecs[k][e][j] is entry e of the
 *                j-th eigenvector of Sigma_k (orthonormal columns)
 *   eigvals      host [K][P], > 0 and non-increasing in j
 *   rank_mode    EPLL_RANK_FIXED: r_k = (int)rank_param in 1..P for every k;
 *                EPLL_RANK_RHO: r_k = smallest r whose leading eigenvalues hold
 *                a fraction rank_param in (0, 1] of the trace.  Eigenvalues
 *                after r_k are replaced by their mean lambda_k; r_k = P keeps
 *                the exact eigenspace form (Eqs. 7-10).
 *   out          receives the handle; free with epll_gmm_free.
 * Host arrays are copied; nothing is retained.  Synchronous.
 * Errors: EPLL_EINVAL on a bad size/value, EPLL_ENOMEM, EPLL_ECUDA.
 */
epll_status epll_gmm_load(int K, int P, const double *weights, const double *eigvecs,
                          const double *eigvals, int rank_mode, double rank_param,
                          epll_gmm **out);

/* Frees the handle and its workspace (synchronises the device). NULL is a no-op. */
void epll_gmm_free(epll_gmm *g);

/*
 * Attaches the balanced search tree of Sec. "Speed-up via a balanced search
 * tree" (built offline, e.g. by collapsing the GMM with Eqs. 17-19) to a
 * model; the handle keeps its own copy.  Nodes are given in breadth-first
 * order, node 0 the root, the children of node v being the consecutive nodes
 * child_begin[v] .. child_begin[v+1]-1 (child_begin[0] = 1, child_begin[n_nodes]
 * = n_nodes); each node is a zero-mean Gaussian in the layout of
 * epll_gmm_load (host weights [n], eigvecs [n][64][64], eigvals [n][64],
 * flat-tailed with the model's rank rule); leaf_component[v] is the model
 * component of a leaf, -1 for an internal node.  Every component must be
 * exactly one leaf, every leaf at the same depth (1..32), no node may have
 * more than 4 children nor children with more than 256 basis columns in all.
 * n_nodes = 0 detaches.  Synchronous.  Errors: EPLL_EINVAL, EPLL_ENOMEM,
 * EPLL_ECUDA.
 */
epll_status epll_gmm_attach_tree(epll_gmm *g, int n_nodes, const double *weights, const double *eigvecs,
                                 const double *eigvals, const int *child_begin, const int *leaf_component);

/* Copies the chosen ranks r_k (host int[K]) and tail eigenvalues lambda_k
 * (host double[K], 0 where r_k = P) out of the handle; either may be NULL. */
epll_status epll_gmm_ranks(const epll_gmm *g, int *ranks, double *lambdas);

/*
 * Restores x from y = A x + w (Algorithm 1 iterated T times, Sec. "Parameter
 * settings"): beta_t = lambda * beta_mult[t] / sigma^2 with
 * lambda = min{N^-1 ||A^T A||_F^2 / ||A||_2^2, 250 sigma_255^2} computed on the
 * device; initialisation x = y for denoising, (A^T A + 0.2 sigma^2/lambda L)^-1
 * A^T y otherwise (FFT for CONV_PERIODIC and CONV_DECIMATE, conjugate
 * gradients for PIXELWISE).
 * Each iteration: per-beta tables (FP64), patch sampling, extraction,
 * projection + Gaussian selection (FP32 SIMT or BF16 tcgen05 with a fused
 * score/argmin epilogue), near-tie rescoring, Wiener patch estimation
 * (Eqs. 15-16), reprojection by overlap-add averaging and the closed-form
 * image update (Eq. 6).
 *   y, x_out     device [H][W]; x_out may alias y (CONV_DECIMATE: y is
 *                [H/factor][W/factor] and must not alias x_out)
 *   H, W         8 <= H, W and H*W <= 2^26
 *   sigma        noise standard deviation in image units, > 0
 *   beta_mult    host [T], > 0 (the paper uses {1, 4, 8, 16, 32}); T in 0..64;
 *                T = 0 runs only the initialisation and returns x0 (beta_mult
 *                may then be NULL)
 *   opt          NULL = defaults
 * Asynchronous on `stream`.  Errors: EPLL_EINVAL, EPLL_ENOMEM, EPLL_ECUDA.
 */
epll_status epll_restore(epll_gmm *g, const float *y, int H, int W,
                         const epll_degradation *deg, float sigma,
                         const double *beta_mult, int T, const epll_options *opt,
                         float *x_out, void *stream);

/* One image of a batch (y, x_out and a are device memory of the current device). */
typedef struct {
    const float *y;  /* H*W observation */
    float *x_out;    /* H*W result; must not alias another job's buffers */
    const float *a;  /* H*W gains for EPLL_PIXELWISE, NULL otherwise */
    int H, W;
    int kind;        /* EPLL_DENOISE, EPLL_PIXELWISE or EPLL_CONV_PERIODIC */
    float sigma;     /* noise standard deviation in image units */
    const float *kernel; /* EPLL_CONV_PERIODIC: host kh*kw blur kernel, copied at every call */
    int kh, kw;
} epll_job;

enum { EPLL_BATCH_SEQUENTIAL = 0, EPLL_BATCH_GRAPH = 1 };

/*
 * Restores a batch of images of uneven size, noise level and degradation
 * (Algorithm 1 for each, as epll_restore; the per-beta tables are per image).
 *   mode  EPLL_BATCH_SEQUENTIAL: one image after the other on `stream`;
 *         EPLL_BATCH_GRAPH: the images are spread over `lanes` contexts (each
 *         with its own tables and workspace, sharing the model) running on
 *         their own streams, and the whole batch is captured once into a CUDA
 *         graph that later calls with the same jobs replay with one launch.
 *         lanes = 0 lets the library tune the batch: on the first call for a
 *         job list it times the graph for 1, 2, 4 and 8 lanes, then, at the
 *         fastest lane count, for the tile shapes of the selection kernel (256
 *         or 128 basis columns per stage) and of the reprojection (1 or 2
 *         image rows per warp), and keeps the fastest combination.
 * The first call for a job list (and any call with a different one) allocates
 * the lanes' workspaces, runs the batch once eagerly and captures the graph;
 * those calls synchronise the device.  Replays are asynchronous on `stream`.
 * Results are identical to epll_restore on each image.
 * Errors: EPLL_EINVAL (any job invalid: nothing is run), EPLL_ENOMEM, EPLL_ECUDA.
 */
epll_status epll_restore_batch(epll_gmm *g, int n, const epll_job *jobs, const double *beta_mult,
                               int T, const epll_options *opt, int mode, int lanes, void *stream);

/* Tile shapes of this handle's kernels: basis columns per stage of the
 * tensor-core selection (256 or 128; 128 keeps four accumulator buffers in
 * flight instead of two) and image rows per warp of the reprojection (1 or
 * 2).  Every shape computes the same restoration (up to
 * the order of FP32 sums); the batch autotuner starts from these values.
 * Defaults 256 and 1.  Errors: EPLL_EINVAL. */
epll_status epll_set_tiles(epll_gmm *g, int tile_bn, int tile_agg);

/* Selection's first pass over the sampled patches (Eq. 14 for every
 * component, Sec. "Complexity via eigenspace implementation") in clusters of
 * two CTAs (enable = 1) that share each tensor-core product (tcgen05
 * cta_group::2, 256 patch rows): each SM then streams half of every basis
 * tile.  Applies with 256-column tiles to the 16-bit forms (FP16, BF16,
 * split BF16); FP8 and 128-column tiles keep one CTA per product.  The
 * selections are the same either way (the products accumulate in the same
 * order).  Errors: EPLL_EINVAL (null handle, enable not 0 or 1). */
epll_status epll_set_cta_pairs(epll_gmm *g, int enable);

/* The configuration the batch autotuner chose for the last tuned job list of
 * this handle (host out, each nullable): lane count (0 if nothing was tuned),
 * selection basis columns per stage (256 or 128) and reprojection image rows
 * per warp (1 or 2).  Errors: EPLL_EINVAL. */
epll_status epll_batch_config(epll_gmm *g, int *lanes, int *tile_bn, int *tile_agg);

/* Same as epll_restore with HOST buffers: y, deg->a (PIXELWISE) and x_out are
 * host pointers; the copies to and from the workspace are part of the call,
 * which returns after x_out is written (synchronises `stream`).  y is H x W
 * ((H/factor) x (W/factor) for CONV_DECIMATE). */
epll_status epll_restore_host(epll_gmm *g, const float *y, int H, int W,
                              const epll_degradation *deg, float sigma,
                              const double *beta_mult, int T, const epll_options *opt,
                              float *x_out, void *stream);

/*
 * One patch step (the first four steps of Algorithm 1) at a given beta, for
 * testing and instrumentation.
 *   xhat         device [H][W], current estimate
 *   beta         > 0 (the paper's beta, i.e. 1/beta is the added variance)
 *   t            iteration index fed to the sampler's counter-based draws
 *   xtilde       device [H][W] out: reprojected patch average (uncovered
 *                pixels copy xhat)
 *   anchors      device int[H*W] out (nullable): sampled anchors (i*W + j of
 *                the top-left pixel), in sampler order
 *   kstar, gap   device int[H*W] / float[H*W] out (nullable): selected
 *                component and top-2 score gap of each sampled patch
 *   forced_k     device int (nullable): per sampled patch, a component that
 *                replaces the selection (teacher forcing)
 *   n_out        host out (nullable): number of sampled patches; when
 *                non-NULL the call synchronises `stream` and returns
 *                EPLL_ETIMEOUT if a bounded device wait gave up
 */
epll_status epll_patch_step(epll_gmm *g, const float *xhat, int H, int W, double beta,
                            const epll_options *opt, int t, float *xtilde, int *anchors,
                            int *kstar, float *gap, const int *forced_k, int *n_out,
                            void *stream);

/*
 * The image estimation step alone (last step of Algorithm 1, Eq. 6 with the
 * constant patch overlap of periodic boundaries), for testing: given the
 * reprojected patch average xtilde,
 *   x = (A^T A + bs I)^-1 (A^T y + bs xtilde),  bs = lambda * beta_mult,
 * with lambda computed from the degradation as in epll_restore.  Pixelwise A
 * (and denoising, a = 1): x = (a y + bs xtilde) / (a^2 + bs) per pixel;
 * CONV_PERIODIC: the same division frequency by frequency (cuFFT);
 * CONV_DECIMATE: A^T A couples the factor^2 frequencies that alias onto one
 * low-resolution frequency through a rank-one block, solved in closed form
 * per block (Woodbury) between full complex FFTs.
 *   y                 device [H][W] ([H/factor][W/factor] for CONV_DECIMATE)
 *   xtilde, x_out     device [H][W]; x_out must not alias y or xtilde
 *   beta_mult         > 0 (the iteration's multiplier m_t)
 * Asynchronous on `stream`.  Errors: EPLL_EINVAL, EPLL_ENOMEM, EPLL_ECUDA.
 */
epll_status epll_image_update(epll_gmm *g, const float *y, const float *xtilde, int H, int W,
                              const epll_degradation *deg, float sigma, double beta_mult, float *x_out,
                              void *stream);

/* Patch sampling alone (for tests): writes the anchors of iteration t to the
 * device buffer `anchors` (capacity H*W) and their count to *n_out (host);
 * synchronises `stream`. */
epll_status epll_sample(int H, int W, const epll_options *opt, int t, int *anchors,
                        int *n_out, void *stream);

/*
 * Patch sampling that allocates nothing on the device (the paper has no
 * counterpart; this is an interface for callers that cannot allocate device
 * memory while they run, e.g. between a pool allocator's fixed reservations or
 * in a loop where cudaMalloc's implicit synchronisation would stall other
 * streams).  Same arguments and output as epll_sample, except that it does not
 * synchronise: it enqueues the sampler on `stream` and returns; *n_out is set
 * on return (the count depends only on H, W and the options).
 * Scratch: a file-scope device array of about 4.2 MB, present on every device
 * that loads the library until the process exits; it serves images of up to
 * 2^20 pixels (larger ones return EPLL_EINVAL).  Every call shares the array
 * and the work it enqueues clears what must start at zero, so calls whose
 * device work overlaps (different streams, no ordering between them) race.
 * Every call looks up the array's device address (cudaGetSymbolAddress) on
 * the current device; the first call on a device may load the library's
 * device code there, so make it before any stream capture.  Arguments are
 * validated as for epll_sample, plus the 2^20-pixel limit.
 * Errors: EPLL_EINVAL, EPLL_ECUDA.
 */
epll_status epll_sample_noalloc(int H, int W, const epll_options *opt, int t, int *anchors,
                                int *n_out, void *stream);

/* Counters of the last epll_restore / epll_patch_step on this handle (host
 * out; synchronises the device): patch evaluations, near-tie rescored
 * patches, and kernel launches issued. */
epll_status epll_last_counters(epll_gmm *g, long long *patch_evals, long long *rescored,
                               long long *launches);

/* Patches that the last epll_restore / epll_patch_step with the proposal
 * selection sent to the exhaustive pass (too little proposal mass or a
 * near-tie among the proposals), summed over its iterations; host out;
 * synchronises the device. */
epll_status epll_last_fallbacks(epll_gmm *g, long long *fallbacks);

/* Instrumentation of the selection kernel (the projection + score contraction,
 * the step that dominates the restoration's arithmetic; with the proposal
 * selection, the fused network kernel instead, whose algorithmic FLOPs are
 * 2 (64*256 + 256*256 + 256*K) per patch).  While enabled, the
 * library records a pair of CUDA events on the call's stream around every
 * launch of that kernel (at most 8192 launches between reads; later launches
 * are not recorded).  epll_profile_read synchronises the device, returns the
 * summed device time in milliseconds, the number of recorded launches and
 * their algorithmic floating-point operations (2 * 64 * sum_k r_k per patch,
 * whatever the arithmetic), then clears the record.  Any output may be NULL. */
epll_status epll_profile_enable(epll_gmm *g, int enable);
epll_status epll_profile_read(epll_gmm *g, double *ms, long long *launches, double *flops);

/*
 * Learned top-m proposal for the Gaussian selection (no counterpart in the
 * paper, which accelerates the selection with a balanced search tree instead;
 * the label it learns is the exact argmin of Eq. 14).  A network
 * 64 -> 256 -> 256 -> K with GELU (erf form) reads a patch's DC-free values
 * z scaled by sqrt(beta); log(1/beta) enters the first layer through a learned
 * per-unit coefficient wb:
 *   h1 = gelu(W1 (sqrt(beta) z) + b1 + log(1/beta) wb),  h2 = gelu(W2 h1 + b2),
 *   logits = W3 h2 + b3.
 * Parameters: one FP32 vector of epll_proposal_size(K) entries in the order
 * W1[256][64], b1[256], wb[256], W2[256][256], b2[256], W3[K][256], b3[K]
 * (matrices row-major [out][in]).  Every forward pass uses W1, W2 and W3
 * rounded to BF16 (round to nearest even) with FP32 biases and FP32
 * accumulation; inference also rounds its layer inputs (sqrt(beta) is applied
 * after the first product: W1 (sqrt(beta) z) = sqrt(beta) (W1 z)) and the
 * hidden activations to BF16.  Training keeps FP32 master weights.
 */
/* Number of parameters for K components (0 if K < 1). */
size_t epll_proposal_size(int K);
/* Creates a network for K in 2..256 components, initialised from `seed`
 * (normal draws scaled by sqrt(2/fan_in), sqrt(1/256) for W3; biases 0).
 * Synchronous.  Errors: EPLL_EINVAL, EPLL_ENOMEM, EPLL_ECUDA. */
epll_status epll_proposal_create(int K, uint64_t seed, epll_proposal **out);
/* Frees the network (synchronises the device).  NULL is a no-op.  Detach it
 * (epll_gmm_attach_proposal with NULL) from every model first. */
void epll_proposal_free(epll_proposal *p);
/* Copies the FP32 master parameters to / from host memory (size entries).
 * set resets the optimiser state.  Synchronous.  Errors: EPLL_EINVAL (NULL, or
 * a non-finite value for set), EPLL_ECUDA. */
epll_status epll_proposal_get(const epll_proposal *p, float *params);
epll_status epll_proposal_set(epll_proposal *p, const float *params);
/*
 * Mean softmax cross-entropy of a batch of B labelled patches and its gradient
 * with respect to the parameters (forward with the BF16-rounded weights,
 * FP32 activations; gradients are those of the rounded weights).
 *   images   device [n_img][H][W] float32 (the patches' source images)
 *   img_idx  device int[n_all]: image of each sample
 *   anchors  device int[n_all]: top-left pixel i*W + j of each 8x8 patch (periodic)
 *   log_ib   device float[n_all]: log(1/beta) of each sample
 *   labels   device int[n_all] in 0..K-1: the exact selection of each sample
 *   sel      device int[B] (nullable): the batch's samples as indices into the
 *            n_all-long arrays; NULL means samples 0..B-1 (then n_all == B)
 *   grad     device float[size] out (nullable)
 *   loss     host float out (nullable); when given, the call synchronises
 *            `stream` and returns EPLL_EINVAL if a sample had an index, anchor,
 *            label or log(1/beta) out of range (such samples contribute nothing)
 * Errors: EPLL_EINVAL, EPLL_ENOMEM, EPLL_ECUDA.
 */
epll_status epll_proposal_grad(epll_proposal *p, const float *images, int n_img, int H, int W,
                               const int *img_idx, const int *anchors, const float *log_ib,
                               const int *labels, const int *sel, int n_all, int B, float *grad,
                               float *loss, void *stream);
/* One AdamW step (beta1 0.9, beta2 0.999, eps 1e-8, decoupled weight decay on
 * W1, W2 and W3 only) on the gradient of the same loss; arguments as
 * epll_proposal_grad; finite lr > 0 and weight_decay >= 0.  The loss is that
 * of the parameters before the step. */
epll_status epll_proposal_train(epll_proposal *p, const float *images, int n_img, int H, int W,
                                const int *img_idx, const int *anchors, const float *log_ib,
                                const int *labels, const int *sel, int n_all, int B, float lr,
                                float weight_decay, float *loss, void *stream);
/* Attaches (p != NULL) or detaches (p == NULL) a network to a model with the
 * same K; topm in 1..min(8, K) proposals per patch; a patch whose proposals
 * hold less than pmin in [0, 1] of the softmax mass is scored exhaustively.
 * The model does not own the network. */
epll_status epll_gmm_attach_proposal(epll_gmm *g, const epll_proposal *p, int topm, float pmin);
/* Runs the attached network (inference kernels) on the patches of xhat
 * (device [H][W]) at anchors (device int[n], NULL = all H*W positions in
 * raster order, n = H*W) for the given beta: cand device int[n][topm] gets
 * the proposed components by decreasing logit (lowest index first on equal
 * logits), pmass device float[n] their softmax mass (nullable).  Asynchronous.
 * Errors: EPLL_EINVAL (no network attached, bad sizes), EPLL_ENOMEM, EPLL_ECUDA. */
epll_status epll_proposal_topm(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                               double beta, int *cand, float *pmass, void *stream);

/* Thread-local message describing the last error of this thread ("" if none). */
const char *epll_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* EPLL_H */
