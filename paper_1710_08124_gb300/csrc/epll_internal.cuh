// Internal declarations of libepll: the model handle, its workspace, the
// per-beta tables, and the kernels' host-side launchers.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cufft.h>

#include <cstdint>
#include <string>

#include "epll.h"

namespace epll {

constexpr int PS = 8;   // patch side
constexpr int PD = 64;  // patch dimension P
constexpr int COL_ALIGN = 8;    // each component's columns are padded to a multiple of this
constexpr int RTOT_ALIGN = 256; // total column count is padded to a multiple of this

// Per-beta quantities of Eq. 14 (flat-tail Gaussian selection) and Eq. 15-16
// (patch estimation), written by the FP64 tables kernel every iteration.
//   score_k(z) = cst_k + t_k |z|^2 + sum_j q_kj c_kj^2,  c_k = Ubar_k^T z
//   cst_k = -2 log w_k + sum_{j<r} log nu_kj + (P - r_k) log nu_kP - cst_0
//   t_k = 1/nu_kP (0 when r_k = P),  q_kj = 1/nu_kj - t_k
//   gw_kj = gamma_kj - gamma_kP,  gp_k = gamma_kP (0 when r_k = P)
// The shared offset cst_0 (component 0's constant) keeps FP32 scores small;
// it does not change the argmin or any gap.  hi/lo pairs hold the FP64 value
// as an unevaluated float sum for the compensated rescoring.
struct Tables {
    float *cst_hi = nullptr, *cst_lo = nullptr;  // [K]
    float *t_hi = nullptr, *t_lo = nullptr;      // [K]
    float *gp = nullptr;                         // [K]
    float *sgn = nullptr;                        // [K]: sign of q_kj (+1 full rank, -1 flat tail)
    float *q_hi = nullptr, *q_lo = nullptr;      // [Rtot]
    float *gw = nullptr;                         // [Rtot]
    float *tmax = nullptr;                       // [1]: max_k 1/min_j nu_kj (error scale)
    float *ibeta = nullptr;                      // [1]: 1/beta of this iteration
    uint16_t *B1 = nullptr;                      // [Rtot][64]: 16-bit Ubar * sqrt|q| (BF16 or FP16), K-major
    uint16_t *Bs = nullptr;                      // [Rtot][64]: BF16 hi part of Ubar * sqrt|q| (split form)
    uint16_t *Bs_lo = nullptr;                   // [Rtot][64]: BF16 remainder (split form)
    uint8_t *B8 = nullptr;                       // [Rtot][64]: E4M3 Ubar * sqrt|q| / s_k
    float *k8s2 = nullptr;                       // [K]: s_k^2 of the E4M3 basis
    float *k8s = nullptr;                        // [K]: s_k
    float *sq = nullptr;                         // [Rtot]: sqrt|q_kj| (0 beyond each rank), the basis scale
};

// Relative score error bound of the split BF16 form (hi*hi + lo*hi + hi*lo):
// a top-2 gap below tau_abs + SPLIT_REL |z|^2 tmax is a near-tie.
constexpr float SPLIT_REL = 4e-5f;
// The same for FP32 dot products of 64 terms.
constexpr float F32_REL = 1e-5f;

// Iterations prepared together (tables of every beta, patch subsets).
constexpr int TB_MAX = 8;

// Tables of batch slot `slot` inside storage laid out slot-major: K-sized
// arrays with stride K, column arrays with stride Rp (Rtot + padding), bases
// with stride Rtot * 64, tmax with stride 1.
__host__ __device__ inline Tables slot_tables(Tables t, int slot, int K, int Rp, int Rtot)
{
    t.cst_hi += (size_t)slot * K; t.cst_lo += (size_t)slot * K;
    t.t_hi += (size_t)slot * K; t.t_lo += (size_t)slot * K;
    t.gp += (size_t)slot * K; t.sgn += (size_t)slot * K;
    t.q_hi += (size_t)slot * Rp; t.q_lo += (size_t)slot * Rp; t.gw += (size_t)slot * Rp;
    t.tmax += slot;
    t.ibeta += slot;
    t.B1 += (size_t)slot * Rtot * 64; t.Bs += (size_t)slot * Rtot * 64; t.Bs_lo += (size_t)slot * Rtot * 64;
    t.B8 += (size_t)slot * Rtot * 64; t.k8s2 += (size_t)slot * K;
    t.k8s += (size_t)slot * K; t.sq += (size_t)slot * Rp;
    return t;
}

// Slots of Workspace::counts after the K bucket counters.
enum { CNT_NFLAG = 0, CNT_ERR = 1, CNT_NFLAG1 = 2 };

struct Workspace {
    size_t capN = 0;
    float *xhat = nullptr, *xtil = nullptr;   // [N]
    float *y = nullptr, *a = nullptr;         // [N], host-buffer entry point only
    int *anchors = nullptr;                   // current iteration's subset: anchors_all + slot * N
    unsigned *mult = nullptr;                 // multiplicity of each anchor in the current subset
    int *anchors_all = nullptr;               // [TB_MAX][N]
    unsigned *mult_all = nullptr;             // [TB_MAX][N]
    size_t sstride = 0;                       // sampler scratch per batch slot (uint32 words)
    int *kstar = nullptr;                     // [N]
    float *gap = nullptr;                     // [N]
    int *flag = nullptr;                      // [N] near-tie list for the compensated rescoring
    int *flag1 = nullptr;                     // [N] near-tie list of a one-term tensor pass
    uint16_t *Z2 = nullptr;                   // [2][zrows][64] split operands of listed rows
    float *zz2 = nullptr;                     // [N] |z|^2 of listed rows
    float *zsc2 = nullptr;                    // [N] squared per-row scale of 8-bit operands
    float *fscore = nullptr;                  // [fcap][K] FP32 scores of listed rows
    size_t fcap = 0;
    int *perm = nullptr;                      // [N] list entries grouped by component
    int4 *items = nullptr;                    // [1 + N/128 + K] estimation work items
    float *zrow = nullptr;                    // [8][N][8] patch estimates: plane u holds patch row u of
                                              // every sampled patch, by its index in the subset
    int *inv = nullptr;                       // [N] index in the subset of a sampled anchor (estimation writes it)
    uint16_t *Zb = nullptr;                   // [2][zrows][64] 16-bit DC-free patches (tensor path)
    size_t zrows = 0;                         // N rounded up to the 128-row tile
    float *zz = nullptr;                      // [N] |z|^2 (tensor path)
    float *mu = nullptr;                      // [N] patch means (split extraction)
    float *cg = nullptr;                      // [4N] CG vectors r, d (two buffers), q
    float *wgt = nullptr;                     // [N] per-pixel overlap weights (`valid` boundary)
    float *red = nullptr;                     // reduction partials
    double *scal = nullptr;                   // [0]: lambda, input of the FP64 per-beta tables
    float *lamf = nullptr;                    // [2]: lambda as an unevaluated float pair (hi, lo)
    unsigned *sampler = nullptr;              // radix-select histograms and state
    int *counts = nullptr;                    // [2K+8] bucket counts/cursors + counters
    long long *ctr = nullptr;                 // [4] device counters: rescored patches
    cufftComplex *Yh = nullptr, *Hh = nullptr, *Xh = nullptr;  // [H][W/2+1]
    float *kern = nullptr;                    // [H][W] wrapped blur kernel
    cufftHandle plan_r2c = 0, plan_c2r = 0;   // the plans of the current size (a cache entry)
    // periodic-blur plans of every size used with this workspace (a batch lane
    // restores several sizes; plans are never created while a graph is captured
    // because the eager run before the capture creates them)
    static constexpr int FFT_CACHE = 8;
    int plan_h[FFT_CACHE] = {}, plan_w[FFT_CACHE] = {};
    cufftHandle plan_fw[FFT_CACHE] = {}, plan_bw[FFT_CACHE] = {};
    int nplans = 0;
    cufftHandle plan_c2c = 0, plan_c2c_low = 0;  // super-resolution: H x W and (H/d) x (W/d)
    int c2cH = 0, c2cW = 0, c2cd = 0;
    // search tree (allocated on first use)
    int *tnode = nullptr;                     // [N] current node of each patch
    int *tcounts = nullptr;                   // [nodes] bucket counters
    int4 *titems = nullptr;                   // work items of a level
    size_t tree_cap = 0;
    int tree_nodes = 0;
    // learned proposal (allocated on first use)
    size_t prop_cap = 0;
    int *cand = nullptr;                      // [N][topm] proposed components
    float *pmass = nullptr;                   // [N] softmax mass of the proposals
    int *pperm = nullptr;                     // [N * topm] pairs grouped by component
    int4 *pitems = nullptr;                   // pair work items
    float *pscore = nullptr;                  // [N * topm] FP32 scores of the pairs
};

struct BatchState;  // lanes, streams and the captured graph of epll_restore_batch

// Search tree attached to a model: its nodes form a model of their own (the
// node Gaussians, flat-tailed with the model's rank rule; tables per beta),
// in breadth-first order with every node's children consecutive.
struct TreeState {
    epll_gmm *tm = nullptr;       // node model (owned)
    int n_nodes = 0, depth = 0;
    int *d_child = nullptr;       // [n_nodes + 1] child ranges
    int *d_leaf = nullptr;        // [n_nodes] component of a leaf, -1 otherwise
    bool owns_arrays = true;      // batch lanes share their handle's child / leaf arrays
    const TreeState *src = nullptr;  // for a lane: the handle's tree it mirrors
    double child_cols_mean = 0;   // mean basis columns of a node's children (instrumentation)
};

}  // namespace epll

struct epll_gmm {
    int K = 0;
    int Rtot = 0;                 // padded total number of basis columns
    int uniform_rank = 0;         // r if every component has rank r, else 0
    int rank_mode = 0;
    double rank_param = 0.0;
    int *h_r = nullptr;           // [K]
    double *h_lam = nullptr;      // [K]
    int *h_roff = nullptr;        // [K+1] column offsets (padded)
    // device model
    int *d_r = nullptr, *d_roff = nullptr, *d_colk = nullptr;   // colk: [Rtot] component of each column (-1: none)
    int4 *d_tileg = nullptr;      // [Rtot / 256] column-group starts of each tile (ragged-rank selection)
    double *d_S = nullptr, *d_w = nullptr, *d_lam = nullptr;     // [K][64], [K], [K]
    float *d_B = nullptr;         // [64][Rtot] Ubar_k concatenated (FP32 rounding of U)
    float *d_Blo = nullptr;       // [64][Rtot] U - B (the FP32 rounding error)
    uint16_t *d_Ub = nullptr;     // [2][Rtot][64] BF16 hi, lo of B transposed (estimation, first product)
    uint16_t *d_U2b = nullptr;    // [2][64][Rtot] BF16 hi, lo of B (estimation, second product)
    epll::Tables tab;             // tables of the current iteration (a slot of tab0)
    epll::Tables tab0;            // storage of TB_MAX iterations' tables
    int Rp = 0;                   // Rtot + column padding
    epll::Workspace ws;
    long long last_evals = 0, last_launches = 0;
    long long launches = 0;
    long long rank_sum = 0;       // sum_k r_k (algorithmic columns)
    // instrumentation of the selection kernel
    bool prof_on = false;
    int prof_n = 0;
    cudaEvent_t *prof_ev = nullptr;   // [2 * PROF_MAX]
    double prof_flops = 0.0;
    // batched restoration: a lane is a context that shares this handle's model
    // arrays and owns its own tables and workspace
    bool lane = false;
    epll::BatchState *batch = nullptr;
    // search tree (owned; see TreeState)
    epll::TreeState *tree = nullptr;
    // learned top-m proposal (not owned)
    const epll_proposal *prop = nullptr;
    int prop_topm = 0;
    float prop_pmin = 0.0f;
    // tile shapes (chosen per lane by the batch autotuner): basis columns per
    // stage of the tensor-core selection (256 or 128), image rows per warp
    // of the reprojection (1 or 2)
    int tile_bn = 256;
    int tile_agg = 1;
    int tc_pair = 0;  // selection first pass in CTA pairs (tcgen05 cta_group::2)
    // second stream: the patch sampler runs on it beside the tables kernels
    // (fork / join through the two events; created on first use)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace epll {

// ---------------------------------------------------------------- error state
void set_error(const std::string &msg);
#define EPLL_CU(call)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            epll::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));        \
            return EPLL_ECUDA;                                                         \
        }                                                                              \
    } while (0)
#define EPLL_LAUNCHED(g)                                                               \
    do {                                                                               \
        ++(g)->launches;                                                               \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess) {                                                       \
            epll::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_));   \
            return EPLL_ECUDA;                                                         \
        }                                                                              \
    } while (0)

// ---------------------------------------------------------------- programmatic dependent launch
// The hot-path kernels are launched with programmatic stream serialization:
// a kernel may be scheduled while its predecessor in the stream finishes, and
// waits at its start (griddepcontrol.wait) until the predecessor has completed
// and its memory is visible; every kernel lets its successor launch as soon as
// all of its own blocks are running (griddepcontrol.launch_dependents), so the
// launch latency and set-up of one kernel overlap the tail of the previous one.
// Launched without the attribute, both instructions have no effect.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter()
{
    pdl_wait();
    pdl_trigger();
}
// Off while the batch issues its lanes: kernels of other lanes' streams could
// then find the SMs held by blocks that launched early and only wait.
inline thread_local bool t_pdl = true;
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = t_pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}

// ---------------------------------------------------------------- launchers
// Each returns EPLL_OK or an error after setting the message.  All enqueue on st.
// Tables of nb iterations at once (slot b: multiplier mult[b], or 1/beta =
// 1/beta_direct when beta_direct > 0).  fmt bit mask: 1 = B1 as BF16,
// 2 = B1 as FP16, 4 = split BF16 basis (Bs, Bs_lo).
epll_status launch_tables(epll_gmm *g, const double *d_lambda, const double *mult, int nb,
                          double sigma2, double beta_direct, int fmt, cudaStream_t st);

// Patch subsets of iterations t0 .. t0+nb-1 into anchors[b * N ...] and
// mult[b * N ...]; *n = patches per iteration.  FULL writes nothing.
epll_status launch_sample(epll_gmm *g, int H, int W, const epll_options &o, int t0, int nb, int *n,
                          int *anchors, unsigned *mult, unsigned *scratch, size_t sstride,
                          cudaStream_t st);
// Scratch words per iteration reserved for the samplers (histograms,
// selection state and per-tile counts of FRAC_TILE anchors); the current
// random-fraction sampler keeps all of it in shared memory, the reservation
// stays part of the workspace layout.
constexpr int FRAC_ITEMS = 8;
constexpr int FRAC_TILE = 256 * FRAC_ITEMS;
constexpr size_t sampler_words(size_t N) { return 1040 + 2 * (N / FRAC_TILE + 2); }
size_t sampler_stride(size_t N);  // = sampler_words(N)
int sample_count(int H, int W, const epll_options &o);
// Argument checks shared by the entry points (set the error message).
epll_status check_options(const epll_options &o, int H, int W);
epll_status check_image(int H, int W);

// Near-tie threshold: gap < tau_abs + tau_rel * |z|^2 * tmax.
epll_status launch_select_fp32(epll_gmm *g, const float *xhat, int H, int W, const int *anchors,
                               int n, float tau_abs, float tau_rel, cudaStream_t st);
epll_status launch_select_tc(epll_gmm *g, const float *xhat, int H, int W, const int *anchors,
                             int n, int precision, float tau_abs, float tau_rel, cudaStream_t st);
// Compensated rescoring of ws.flag (count in counts[2K + CNT_NFLAG]).  With
// split_scores the candidate scores come from the split-BF16 tensor pass.
epll_status launch_rescore(epll_gmm *g, const float *xhat, int H, int W, const int *anchors,
                           int n, bool split_scores, float tau_abs, cudaStream_t st);
epll_status launch_dump_split(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                              cudaStream_t st);
epll_status launch_split_pass(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                              const int *flag1, const int *nflag1, float tau_abs, cudaStream_t st);
// Learned top-m proposal + exact FP32 rescoring of the proposals; undecided
// patches go through launch_split_pass.  Leaves kstar/gap of every row and the
// near-tie list of the split pass for launch_rescore.
epll_status launch_select_proposal(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                                   float tau_abs, cudaStream_t st);
// Proposal network alone: top-m components and their softmax mass per patch
// (1/beta read from the device scalar ibeta).
epll_status launch_proposal_topm(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                                 const float *ibeta, cudaStream_t st);
// Operand rows of n sampled patches (csrc/k_extract.cu): row i is patch i, or
// patch rowmap[i] of a device list with device count *n_dev; fmt 1 BF16,
// 2 FP16 (split: hi into Zhi, lo into Zlo), 3 E4M3 with the squared row scale
// in zsc2; |z|^2 into zz, the means into mu (nullable); Zf (nullable) an
// FP16 copy of the rows beside the fmt rows.
epll_status launch_extract(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                           const int *rowmap, const int *n_dev, int fmt, int split, uint16_t *Zhi, uint16_t *Zlo,
                           float *zz, float *zsc2, float *mu, cudaStream_t st, uint16_t *Zf = nullptr);
// Split BF16 (hi, lo) DC-free patches into ws.Zb's two halves (rows padded
// to 128 with zeros), |z|^2 into ws.zz and the patch means into ws.mu.
epll_status launch_extract_split(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                                 cudaStream_t st);
// Candidate pairs (csrc/k_mlp.cu): ws.cand holds m candidate components per
// entry (negative: absent); entry f is patch f, or patch list[f] of a device
// list with device count *nlist.  launch_pair_scores groups the pairs by
// component and writes their split-BF16 scores of Eq. 14 to ws.pscore;
// launch_cand_combine writes each listed patch's best rescored candidate to
// kstar / gap and appends the patch to flag (count nflag) when its top-2 gap
// is within the split form's error bound or its first candidate is absent.
epll_status ensure_prop_ws(epll_gmm *g, int n);
epll_status launch_pair_scores(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n, int m,
                               const int *list, const int *nlist, cudaStream_t st);
epll_status launch_cand_combine(epll_gmm *g, int n, int m, const int *list, const int *nlist, float tau_abs,
                                int *flag, int *nflag, cudaStream_t st);
// Counting sort of n keys (components; negative keys are left out) into perm
// and estimation work items; with n_dev the key count is min(n, mult * *n_dev).
epll_status group_by_component(epll_gmm *g, const int *keys, int n, int *perm, int4 *items, cudaStream_t st,
                               const int *n_dev = nullptr, int mult = 1);
// Same for keys in 0..K-1 with an explicit [K] counter array.
epll_status group_by_key(epll_gmm *g, const int *keys, int n, int K, int *counts, int *perm, int4 *items,
                         cudaStream_t st, const int *n_dev = nullptr, int mult = 1);
// Selection down the search tree (csrc/k_tree.cu): writes kstar and the
// smallest sibling gap on each patch's path.
epll_status launch_select_tree(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                               cudaStream_t st);
// A context sharing g's model arrays with its own tables (csrc/batch.cu).
epll_gmm *make_lane(const epll_gmm *g);
void free_tree(epll_gmm *g);
inline int *cnt(epll_gmm *g, int slot) { return g->ws.counts + 2 * g->K + slot; }
epll_status launch_estimate(epll_gmm *g, const float *xhat, int H, int W, const int *anchors,
                            int n, cudaStream_t st);
// Same on the tensor cores in the split BF16 form (csrc/k_estimate_tc.cu).
// With reuse, the split operands and means the selection extracted (ws.Zb,
// ws.mu) are copied instead of gathering the patches from the image again.
epll_status launch_estimate_tc(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                               bool reuse, cudaStream_t st);
// Reprojection.  When y != nullptr the pixelwise image update is fused
// (xout = (a y + bs xt)/(a^2 + bs), bs = lambda*mult with lambda = lamf[0];
// a == nullptr means a = 1), otherwise xtilde is written to xout.
// weighted: bs is multiplied by each pixel's patch count / P (Eq. 6 with the
// `valid` boundary); wout (nullable) receives that weight.
epll_status launch_aggregate(epll_gmm *g, const float *xhat, int H, int W, const unsigned *mult,
                             const float *y, const float *a, const float *lamf, double bmult,
                             float *xout, cudaStream_t st, int weighted = 0, float *wout = nullptr);
// Image update of a periodic blur with per-pixel overlap weights ws.wgt
// (`valid` boundary): iters conjugate-gradient iterations on
// (H^T H + bs diag(w)) x = H^T y + bs w xtil from x = xtil (ws.xtil -> ws.xhat).
epll_status cgw_update(epll_gmm *g, int H, int W, double bmult, int iters, cudaStream_t st);

// Image-domain steps (k_image.cu)
epll_status launch_lambda(epll_gmm *g, int kind, const float *a, int H, int W, double sigma,
                          cudaStream_t st, int d = 1);   // writes ws.scal[0] and ws.lamf
// plans, Hh, Yh; the kh x kw kernel is host memory, or device memory when kernel_dev
epll_status fft_prepare(epll_gmm *g, const float *kernel, int kh, int kw, const float *y,
                        int H, int W, cudaStream_t st, bool kernel_dev = false);
epll_status fft_init(epll_gmm *g, int H, int W, double sigma, cudaStream_t st);    // ws.xhat
epll_status fft_update(epll_gmm *g, int H, int W, double bmult, cudaStream_t st);  // ws.xtil -> ws.xhat
// Super-resolution (blur, then decimation by d): full complex transforms of
// the kernel and of the low-resolution observation, the initialisation and
// the image update (ws.xtil -> ws.xhat), each solved per aliasing block.
epll_status sr_prepare(epll_gmm *g, const float *kernel_host, int kh, int kw, const float *ylow, int H, int W,
                       int d, cudaStream_t st);
epll_status sr_init(epll_gmm *g, int H, int W, int d, double sigma, cudaStream_t st);
epll_status sr_update(epll_gmm *g, int H, int W, int d, double bmult, cudaStream_t st);
epll_status cg_init(epll_gmm *g, const float *a, const float *y, int H, int W, double sigma,
                    int iters, cudaStream_t st);  // ws.xhat (one cluster launch)
void cg_setup();     // picks the CG kernel's cluster size; call outside stream capture
void group_setup();  // the same for the grouping kernel
void sampler_setup();  // the same for the random-fraction sampler
// x = (a y + bs xt)/(a^2 + bs), bs = lambda * bmult (a == nullptr: a = 1)
epll_status launch_pixel_update(epll_gmm *g, const float *a, const float *y, const float *xt, int H, int W,
                                double bmult, float *x, cudaStream_t st);

// Training product C[m * ldc + n] = sum_k A[m sam + k sak] B[k sbk + n sbn]
// (FP32 in and out) on the tensor cores, split BF16 operands; long
// reductions are split across CTAs into `partial` (capacity in floats).
// N <= 256.  err is set if a bounded wait gave up.
epll_status gemm_tc(const float *A, long sam, long sak, const float *B, long sbk, long sbn, float *C, int ldc, int M,
                    int N, int Kd, float *partial, size_t partial_cap, int *err, cudaStream_t st);

epll_status ensure_workspace(epll_gmm *g, size_t N);
epll_status fail(epll_status s, const std::string &msg);
cudaError_t alloc_tables(epll_gmm *g);
void free_batch(epll_gmm *g);
// One restoration on g's workspace and tables (no allocation, no synchronisation).
// kernel_dev: deg->kernel (CONV_PERIODIC) is device memory (batch lanes).
epll_status run_restore(epll_gmm *g, const float *y, const float *a, int H, int W,
                        const epll_degradation *deg, float sigma, const double *beta_mult, int T,
                        const epll_options &o, cudaStream_t st, bool kernel_dev = false);
epll_status check_restore_args(epll_gmm *g, const float *y, int H, int W, const epll_degradation *deg,
                               float sigma, const double *beta_mult, int T, const epll_options &o,
                               const float *x_out);

// Selection-kernel instrumentation (no-ops unless enabled).
constexpr int PROF_MAX = 8192;
void prof_begin(epll_gmm *g, cudaStream_t st);
// flops_per_row < 0: the selection GEMM's 2 * 64 * sum_k r_k
void prof_end(epll_gmm *g, cudaStream_t st, int n, double flops_per_row = -1.0);

}  // namespace epll
