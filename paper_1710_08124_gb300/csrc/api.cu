// C ABI of libepll: model loading (flat-tail preparation), workspace
// management and the restoration loop (Algorithm 1 iterated over the beta
// schedule of Sec. "Parameter settings").
#include "epll_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace epll {

void prof_begin(epll_gmm *g, cudaStream_t st)
{
    if (g->prof_on && g->prof_n < PROF_MAX) cudaEventRecord(g->prof_ev[2 * g->prof_n], st);
}
void prof_end(epll_gmm *g, cudaStream_t st, int n, double flops_per_row)
{
    if (g->prof_on && g->prof_n < PROF_MAX) {
        cudaEventRecord(g->prof_ev[2 * g->prof_n + 1], st);
        g->prof_flops += (flops_per_row >= 0.0 ? flops_per_row : 2.0 * PD * (double)g->rank_sum) * (double)n;
        ++g->prof_n;
    }
}

// BF16 of a float, rounded to nearest even (NaN kept quiet), and back.
static uint16_t bf16_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
static float bf16_value(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }

epll_status fail(epll_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

template <typename T>
static cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * count);
}

static void free_workspace(Workspace &ws)
{
    void *ptrs[] = {ws.xhat, ws.xtil, ws.y, ws.a, ws.anchors_all, ws.mult_all, ws.kstar, ws.gap,
                    ws.flag, ws.flag1, ws.Z2, ws.zz2, ws.zsc2, ws.fscore,
                    ws.perm, ws.items, ws.zrow, ws.inv, ws.Zb, ws.zz, ws.mu, ws.cg, ws.wgt, ws.red, ws.scal, ws.lamf,
                    ws.sampler, ws.counts, ws.ctr, ws.Yh, ws.Hh, ws.Xh, ws.kern,
                    ws.cand, ws.pmass, ws.pperm, ws.pitems, ws.pscore, ws.tnode, ws.tcounts, ws.titems};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < ws.nplans; ++i) {
        cufftDestroy(ws.plan_fw[i]);
        cufftDestroy(ws.plan_bw[i]);
    }
    if (ws.plan_c2c) cufftDestroy(ws.plan_c2c);
    if (ws.plan_c2c_low) cufftDestroy(ws.plan_c2c_low);
    ws = Workspace();
}

epll_status ensure_workspace(epll_gmm *g, size_t N)
{
    Workspace &ws = g->ws;
    if (N <= ws.capN) return EPLL_OK;
    EPLL_CU(cudaDeviceSynchronize());
    free_workspace(ws);
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(dalloc(&ws.xhat, N)); A(dalloc(&ws.xtil, N)); A(dalloc(&ws.y, N)); A(dalloc(&ws.a, N));
    A(dalloc(&ws.anchors_all, TB_MAX * N)); A(dalloc(&ws.mult_all, TB_MAX * N));
    A(dalloc(&ws.kstar, N)); A(dalloc(&ws.gap, N));
    A(dalloc(&ws.flag, N)); A(dalloc(&ws.flag1, N)); A(dalloc(&ws.perm, N)); A(dalloc(&ws.zrow, N * PD)); A(dalloc(&ws.inv, N));
    A(dalloc(&ws.items, 2 + N / 128 + (size_t)g->K));
    const size_t zrows = (N + 127) / 128 * 128;
    A(dalloc(&ws.Zb, 2 * zrows * PD)); A(dalloc(&ws.zz, N)); A(dalloc(&ws.mu, N));
    A(dalloc(&ws.Z2, 2 * zrows * PD)); A(dalloc(&ws.zz2, N)); A(dalloc(&ws.zsc2, N));
    // FP32 scores of near-tie rows: at most this many rows per rescoring pass
    size_t fcap = (size_t)1 << 26;
    fcap /= (size_t)g->K;
    if (fcap < 4096) fcap = 4096;
    if (fcap > N) fcap = N;
    A(dalloc(&ws.fscore, fcap * (size_t)g->K)); A(dalloc(&ws.cg, 4 * N)); A(dalloc(&ws.wgt, N));
    A(dalloc(&ws.red, 4096)); A(dalloc(&ws.scal, 16)); A(dalloc(&ws.lamf, 16));
    const size_t sstride = sampler_stride(N);
    A(dalloc(&ws.sampler, TB_MAX * sstride));
    A(dalloc(&ws.counts, 2 * (size_t)g->K + 8)); A(dalloc(&ws.ctr, 4));
    A(dalloc(&ws.Yh, N)); A(dalloc(&ws.Hh, N)); A(dalloc(&ws.Xh, N)); A(dalloc(&ws.kern, N));
    if (e != cudaSuccess) {
        free_workspace(ws);
        cudaGetLastError();
        return fail(EPLL_ENOMEM, std::string("workspace allocation: ") + cudaGetErrorString(e));
    }
    ws.capN = N;
    ws.zrows = zrows;
    ws.fcap = fcap;
    ws.sstride = sstride;
    ws.anchors = ws.anchors_all;
    ws.mult = ws.mult_all;
    EPLL_CU(cudaMemset(ws.ctr, 0, sizeof(long long) * 4));
    EPLL_CU(cudaMemset(ws.counts, 0, sizeof(int) * (2 * (size_t)g->K + 8)));
    return EPLL_OK;
}

// Per-beta tables of TB_MAX iterations, slot-major (see slot_tables).
cudaError_t alloc_tables(epll_gmm *g)
{
    const int K = g->K, R = g->Rtot, Rp = g->Rp;
    Tables &T0 = g->tab0;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(dalloc(&T0.cst_hi, TB_MAX * K)); A(dalloc(&T0.cst_lo, TB_MAX * K)); A(dalloc(&T0.t_hi, TB_MAX * K));
    A(dalloc(&T0.t_lo, TB_MAX * K)); A(dalloc(&T0.gp, TB_MAX * K)); A(dalloc(&T0.sgn, TB_MAX * K));
    A(dalloc(&T0.q_hi, (size_t)TB_MAX * Rp)); A(dalloc(&T0.q_lo, (size_t)TB_MAX * Rp));
    A(dalloc(&T0.gw, (size_t)TB_MAX * Rp));
    A(dalloc(&T0.tmax, TB_MAX)); A(dalloc(&T0.ibeta, TB_MAX));
    A(dalloc(&T0.B1, (size_t)TB_MAX * R * PD));
    A(dalloc(&T0.Bs, (size_t)TB_MAX * R * PD)); A(dalloc(&T0.Bs_lo, (size_t)TB_MAX * R * PD));
    A(dalloc(&T0.B8, (size_t)TB_MAX * R * PD)); A(dalloc(&T0.k8s2, TB_MAX * K));
    A(dalloc(&T0.k8s, TB_MAX * K)); A(dalloc(&T0.sq, (size_t)TB_MAX * Rp));
    if (e != cudaSuccess) return e;
    A(cudaMemset(T0.q_hi, 0, sizeof(float) * (size_t)TB_MAX * Rp));
    A(cudaMemset(T0.q_lo, 0, sizeof(float) * (size_t)TB_MAX * Rp));
    A(cudaMemset(T0.gw, 0, sizeof(float) * (size_t)TB_MAX * Rp));
    A(cudaMemset(T0.sq, 0, sizeof(float) * (size_t)TB_MAX * Rp));
    A(cudaMemset(T0.B1, 0, sizeof(uint16_t) * (size_t)TB_MAX * R * PD));
    A(cudaMemset(T0.Bs, 0, sizeof(uint16_t) * (size_t)TB_MAX * R * PD));
    A(cudaMemset(T0.Bs_lo, 0, sizeof(uint16_t) * (size_t)TB_MAX * R * PD));
    A(cudaMemset(T0.B8, 0, (size_t)TB_MAX * R * PD));
    g->tab = slot_tables(T0, 0, K, Rp, R);
    return e;
}

static void free_tables(epll_gmm *g)
{
    void *ptrs[] = {g->tab0.cst_hi, g->tab0.cst_lo, g->tab0.t_hi, g->tab0.t_lo, g->tab0.gp, g->tab0.sgn,
                    g->tab0.q_hi, g->tab0.q_lo, g->tab0.gw, g->tab0.tmax, g->tab0.ibeta, g->tab0.B1, g->tab0.Bs,
                    g->tab0.Bs_lo, g->tab0.B8, g->tab0.k8s2, g->tab0.k8s, g->tab0.sq};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    g->tab0 = Tables();
    g->tab = Tables();
}


void free_tree(epll_gmm *g)
{
    TreeState *tr = g->tree;
    if (!tr) return;
    if (tr->tm) epll_gmm_free(tr->tm);
    if (tr->owns_arrays) {
        if (tr->d_child) cudaFree(tr->d_child);
        if (tr->d_leaf) cudaFree(tr->d_leaf);
    }
    delete tr;
    g->tree = nullptr;
}

static void free_model(epll_gmm *g)
{
    free_batch(g);
    free_tree(g);
    free_tables(g);
    if (g->lane) return;  // lanes share the model arrays of their handle
    void *ptrs[] = {g->d_r, g->d_roff, g->d_colk, g->d_S, g->d_w, g->d_lam, g->d_B, g->d_Blo, g->d_Ub, g->d_U2b,
                    g->d_tileg};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete[] g->h_r;
    delete[] g->h_lam;
    delete[] g->h_roff;
    if (g->prof_ev) {
        for (int i = 0; i < 2 * PROF_MAX; ++i) cudaEventDestroy(g->prof_ev[i]);
        delete[] g->prof_ev;
    }
}

epll_status check_options(const epll_options &o, int H, int W)
{
    if (o.precision < EPLL_FP32 || o.precision > EPLL_AUTO)
        return fail(EPLL_EINVAL, "options.precision must be EPLL_FP32, _BF16, _FP16, _BF16X3, _FP8 or _AUTO");
    if (!(std::isfinite(o.tie_gap)))
        return fail(EPLL_EINVAL, "options.tie_gap must be finite");
    if (o.subset == EPLL_SUBSET_FRACTION) {
        if (!(o.subset_param > 0.0 && o.subset_param <= 1.0))
            return fail(EPLL_EINVAL, "options.subset_param: fraction must be in (0, 1]");
    } else if (o.subset == EPLL_SUBSET_JITTER || o.subset == EPLL_SUBSET_REGULAR) {
        int s = (int)o.subset_param;
        if ((double)s != o.subset_param || s < 1 || s > PS)
            return fail(EPLL_EINVAL, "options.subset_param: grid spacing must be an integer in 1..8");
        (void)H; (void)W;
    } else if (o.subset != EPLL_SUBSET_ALL && o.subset != EPLL_SUBSET_VALID) {
        return fail(EPLL_EINVAL, "options.subset must be EPLL_SUBSET_ALL, _FRACTION, _JITTER, _REGULAR or _VALID");
    }
    if (o.cg_iters < 0 || o.cg_iters > 100000) return fail(EPLL_EINVAL, "options.cg_iters out of range");
    if (o.select != EPLL_SELECT_EXHAUSTIVE && o.select != EPLL_SELECT_PROPOSAL && o.select != EPLL_SELECT_TREE)
        return fail(EPLL_EINVAL, "options.select must be EPLL_SELECT_EXHAUSTIVE, _PROPOSAL or _TREE");
    return EPLL_OK;
}

static epll_status check_select(const epll_gmm *g, const epll_options &o)
{
    if (o.select == EPLL_SELECT_PROPOSAL && !g->prop)
        return fail(EPLL_EINVAL, "options.select is EPLL_SELECT_PROPOSAL but no proposal network is attached");
    if (o.select == EPLL_SELECT_TREE && !g->tree)
        return fail(EPLL_EINVAL, "options.select is EPLL_SELECT_TREE but no search tree is attached");
    return EPLL_OK;
}

epll_status check_image(int H, int W)
{
    if (H < PS || W < PS) return fail(EPLL_EINVAL, "image must be at least 8 x 8");
    if ((long long)H * W > (1LL << 26)) return fail(EPLL_EINVAL, "image larger than 2^26 pixels");
    return EPLL_OK;
}

// The arithmetic EPLL_AUTO stands for: the FP16 one-term pass with FP32
// candidate rescoring where the projection is long enough for the pass to
// save more than its candidates cost (uniform ranks of 32 and more), the
// split BF16 pass otherwise.
static int eff_precision(const epll_gmm *g, const epll_options &o)
{
    if (o.precision != EPLL_AUTO) return o.precision;
    return g->uniform_rank >= 32 ? EPLL_FP16 : EPLL_BF16X3;
}

// Near-tie threshold tau_abs + tau_rel |z|^2 max 1/nu.  tau_rel bounds the
// relative score error of each arithmetic (twice the largest error observed
// on the synthetic prior, rounded up): FP32 dot products of 64 terms; FP16 /
// BF16 operand rounding (2^-11 / 2^-8 per operand); E4M3 operands with
// per-component / per-patch scales (2^-4 per operand; 4.4e-2 measured); the split BF16 form
// (residual error of order 2^-16; at most 8e-6 relative measured).
static void thresholds(const epll_options &o, int precision, float *tau_abs, float *tau_rel)
{
    *tau_abs = o.tie_gap >= 0.0f ? o.tie_gap : 1e-3f;
    switch (precision) {
    case EPLL_BF16: *tau_rel = 1e-2f; break;
    case EPLL_FP16: *tau_rel = 1.5e-3f; break;
    case EPLL_BF16X3: *tau_rel = 4e-5f; break;
    case EPLL_FP8: *tau_rel = 1e-1f; break;
    default: *tau_rel = F32_REL; break;
    }
}

// Bases the tables kernel writes for each arithmetic (bit mask, see launch_tables).
static int basis_format(const epll_options &o, int precision)
{
    if (o.select == EPLL_SELECT_PROPOSAL) return 4;  // exhaustive fallback: split BF16 pass
    if (o.select == EPLL_SELECT_TREE) return 0;      // the node model carries the bases
    switch (precision) {
    case EPLL_BF16: return 1 | 4;
    case EPLL_FP16: return 2 | 4;
    case EPLL_BF16X3: return 4;
    case EPLL_FP8: return 8 | 4;
    default: return 0;
    }
}

// Per-beta tables and patch subsets of iterations t0 .. t0+nb-1 (one batch):
// the sampler runs on the handle's second stream while the tables kernels
// run on st, and st waits for it (batch lanes, the full set and small images
// run both on st).
static epll_status prepare_batch(epll_gmm *g, int H, int W, const epll_options &o, int t0, int nb,
                                 const double *d_lambda, const double *mult, double sigma2,
                                 double beta_direct, int *n, cudaStream_t st)
{
    Workspace &ws = g->ws;
    epll_status s;
    if (g->lane || o.subset == EPLL_SUBSET_ALL || (size_t)H * W < ((size_t)1 << 16)) {
        // one stream: a batch lane runs beside other lanes already (forks inside
        // the captured batch graph cost more than they overlap), the full set
        // launches no sampler, and a small image's sampler is shorter than a fork
        if ((s = launch_tables(g, d_lambda, mult, nb, sigma2, beta_direct, basis_format(o, eff_precision(g, o)), st)))
            return s;
        if (o.select == EPLL_SELECT_TREE &&
            (s = launch_tables(g->tree->tm, d_lambda, mult, nb, sigma2, beta_direct, 4, st)))
            return s;
        return launch_sample(g, H, W, o, t0, nb, n, ws.anchors_all, ws.mult_all, ws.sampler, ws.sstride, st);
    }
    if (!g->aux) {
        EPLL_CU(cudaStreamCreateWithFlags(&g->aux, cudaStreamNonBlocking));
        EPLL_CU(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
        EPLL_CU(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming));
    }
    EPLL_CU(cudaEventRecord(g->ev_fork, st));
    EPLL_CU(cudaStreamWaitEvent(g->aux, g->ev_fork, 0));
    if ((s = launch_sample(g, H, W, o, t0, nb, n, ws.anchors_all, ws.mult_all, ws.sampler, ws.sstride, g->aux)))
        return s;
    EPLL_CU(cudaEventRecord(g->ev_join, g->aux));
    if ((s = launch_tables(g, d_lambda, mult, nb, sigma2, beta_direct, basis_format(o, eff_precision(g, o)), st)))
        return s;
    if (o.select == EPLL_SELECT_TREE &&
        (s = launch_tables(g->tree->tm, d_lambda, mult, nb, sigma2, beta_direct, 4, st)))
        return s;
    EPLL_CU(cudaStreamWaitEvent(st, g->ev_join, 0));
    return EPLL_OK;
}

// Points the current-iteration views (tables, subset) at batch slot b.
static void use_slot(epll_gmm *g, int b, size_t N)
{
    g->tab = slot_tables(g->tab0, b, g->K, g->Rp, g->Rtot);
    if (g->tree) {
        epll_gmm *tm = g->tree->tm;
        tm->tab = slot_tables(tm->tab0, b, tm->K, tm->Rp, tm->Rtot);
    }
    g->ws.anchors = g->ws.anchors_all + (size_t)b * N;
    g->ws.mult = g->ws.mult_all + (size_t)b * N;
}

// One patch step on prepared tables/subset: selection, rescoring, estimation.
// The reprojection is left to the caller (it may be fused with the image update).
static epll_status patch_phase(epll_gmm *g, const float *xhat, int H, int W, const epll_options &o,
                               int n, const int *forced_k, cudaStream_t st)
{
    Workspace &ws = g->ws;
    epll_status s;
    const int *anchors = o.subset == EPLL_SUBSET_ALL ? nullptr : ws.anchors;
    const int prec = eff_precision(g, o);
    float tau_abs, tau_rel;
    thresholds(o, prec, &tau_abs, &tau_rel);
    if (o.select == EPLL_SELECT_TREE) {
        if ((s = launch_select_tree(g, xhat, H, W, anchors, n, st))) return s;
    } else if (o.select == EPLL_SELECT_PROPOSAL) {
        if ((s = launch_select_proposal(g, xhat, H, W, anchors, n, tau_abs, st))) return s;
    } else if (prec != EPLL_FP32) {
        if ((s = launch_select_tc(g, xhat, H, W, anchors, n, prec, tau_abs, tau_rel, st))) return s;
    } else {
        if ((s = launch_select_fp32(g, xhat, H, W, anchors, n, tau_abs, tau_rel, st))) return s;
    }
    const bool split_scores = o.select == EPLL_SELECT_PROPOSAL || prec != EPLL_FP32;
    if (o.select != EPLL_SELECT_TREE &&
        (s = launch_rescore(g, xhat, H, W, anchors, n, split_scores, tau_abs, st)))
        return s;
    if (forced_k)
        EPLL_CU(cudaMemcpyAsync(ws.kstar, forced_k, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    // the FP32 form keeps the SIMT estimate (FP32 parity with the oracle);
    // the reduced-precision forms use the split-BF16 tensor-core estimate
    if (prec == EPLL_FP32 && o.select == EPLL_SELECT_EXHAUSTIVE) {
        if ((s = launch_estimate(g, xhat, H, W, anchors, n, st))) return s;
    } else {
        // the split and FP16 passes, the proposal and the tree leave every
        // patch's split operands and mean in ws.Zb / ws.mu
        const bool reuse = o.select != EPLL_SELECT_EXHAUSTIVE || prec == EPLL_BF16X3 || prec == EPLL_FP16;
        if ((s = launch_estimate_tc(g, xhat, H, W, anchors, n, reuse, st))) return s;
    }
    g->last_evals += n;
    return EPLL_OK;
}

epll_status run_restore(epll_gmm *g, const float *y, const float *a, int H, int W,
                               const epll_degradation *deg, float sigma, const double *beta_mult,
                               int T, const epll_options &o, cudaStream_t st, bool kernel_dev)
{
    Workspace &ws = g->ws;
    const int kind = deg ? deg->kind : EPLL_DENOISE;
    epll_status s;
    g->launches = 0;
    g->last_evals = 0;
    EPLL_CU(cudaMemsetAsync(ws.ctr, 0, sizeof(long long) * 4, st));
    EPLL_CU(cudaMemsetAsync(cnt(g, CNT_ERR), 0, sizeof(int), st));
    const int d = kind == EPLL_CONV_DECIMATE ? deg->factor : 1;
    if (kind == EPLL_CONV_PERIODIC) {
        if ((s = fft_prepare(g, deg->kernel, deg->kh, deg->kw, y, H, W, st, kernel_dev))) return s;
    } else if (kind == EPLL_CONV_DECIMATE) {
        if ((s = sr_prepare(g, deg->kernel, deg->kh, deg->kw, y, H, W, d, st))) return s;
    }
    if ((s = launch_lambda(g, kind, a, H, W, sigma, st, d))) return s;
    if (kind == EPLL_DENOISE) {
        EPLL_CU(cudaMemcpyAsync(ws.xhat, y, sizeof(float) * (size_t)H * W, cudaMemcpyDeviceToDevice, st));
    } else if (kind == EPLL_CONV_PERIODIC) {
        if ((s = fft_init(g, H, W, sigma, st))) return s;
    } else if (kind == EPLL_CONV_DECIMATE) {
        if ((s = sr_init(g, H, W, d, sigma, st))) return s;
    } else {
        if ((s = cg_init(g, a, y, H, W, sigma, o.cg_iters, st))) return s;
    }
    const double s2 = (double)sigma * sigma;
    const size_t N = (size_t)H * W;
    size_t nbmax = ((size_t)1 << 23) / N;
    if (nbmax < 1) nbmax = 1;
    if (nbmax > (size_t)TB_MAX) nbmax = TB_MAX;
    int n = 0;
    for (int t = 0; t < T; ++t) {
        const int b = (int)(t % nbmax);
        if (b == 0) {
            const int nb = (int)std::min<size_t>(nbmax, (size_t)(T - t));
            if ((s = prepare_batch(g, H, W, o, t, nb, ws.scal, beta_mult + t, s2, 0.0, &n, st))) return s;
        }
        use_slot(g, b, N);
        if ((s = patch_phase(g, ws.xhat, H, W, o, n, nullptr, st))) return s;
        const unsigned *mult = o.subset == EPLL_SUBSET_ALL ? nullptr : ws.mult;
        const bool valid = o.subset == EPLL_SUBSET_VALID;
        if (kind == EPLL_CONV_PERIODIC || kind == EPLL_CONV_DECIMATE) {
            if ((s = launch_aggregate(g, ws.xhat, H, W, mult, nullptr, nullptr, ws.lamf, 0.0, ws.xtil, st, 0,
                                      valid ? ws.wgt : nullptr)))
                return s;
            if (valid) {
                if ((s = cgw_update(g, H, W, beta_mult[t], o.cg_iters, st))) return s;
            } else if (kind == EPLL_CONV_PERIODIC) {
                if ((s = fft_update(g, H, W, beta_mult[t], st))) return s;
            } else {
                if ((s = sr_update(g, H, W, d, beta_mult[t], st))) return s;
            }
        } else {
            if ((s = launch_aggregate(g, ws.xhat, H, W, mult, y, kind == EPLL_PIXELWISE ? a : nullptr,
                                      ws.lamf, beta_mult[t], ws.xhat, st, valid ? 1 : 0)))
                return s;
        }
    }
    g->last_launches = g->launches;
    return EPLL_OK;
}

epll_status check_restore_args(epll_gmm *g, const float *y, int H, int W,
                                      const epll_degradation *deg, float sigma,
                                      const double *beta_mult, int T, const epll_options &o,
                                      const float *x_out)
{
    if (!g) return fail(EPLL_EINVAL, "null model handle");
    if (!y || !x_out) return fail(EPLL_EINVAL, "null image pointer");
    epll_status s;
    if ((s = check_image(H, W))) return s;
    if (!(sigma > 0.0f) || !std::isfinite(sigma)) return fail(EPLL_EINVAL, "sigma must be positive");
    if (T < 0 || T > 64 || (T > 0 && !beta_mult))
        return fail(EPLL_EINVAL, "beta schedule must have 0..64 entries");
    for (int t = 0; t < T; ++t)
        if (!(beta_mult[t] > 0.0) || !std::isfinite(beta_mult[t]))
            return fail(EPLL_EINVAL, "beta multipliers must be positive");
    if ((s = check_options(o, H, W))) return s;
    if ((s = check_select(g, o))) return s;
    if (deg) {
        if (deg->kind == EPLL_PIXELWISE) {
            if (!deg->a) return fail(EPLL_EINVAL, "PIXELWISE degradation needs gains a");
        } else if (deg->kind == EPLL_CONV_PERIODIC || deg->kind == EPLL_CONV_DECIMATE) {
            if (!deg->kernel || deg->kh < 1 || deg->kw < 1 || deg->kh > H || deg->kw > W)
                return fail(EPLL_EINVAL, "blur kernel must be 1..H x 1..W");
            if (deg->kind == EPLL_CONV_DECIMATE &&
                (deg->factor < 1 || deg->factor > 8 || H % deg->factor || W % deg->factor))
                return fail(EPLL_EINVAL, "CONV_DECIMATE factor must be in 1..8 and divide H and W");
            if (deg->kind == EPLL_CONV_DECIMATE && o.subset == EPLL_SUBSET_VALID)
                return fail(EPLL_EUNSUPPORTED, "the VALID boundary is not served with CONV_DECIMATE");
            double sum = 0.0;
            for (int q = 0; q < deg->kh * deg->kw; ++q) {
                if (!std::isfinite(deg->kernel[q])) return fail(EPLL_EINVAL, "kernel is not finite");
                sum += deg->kernel[q];
            }
            if (!(sum > 0.0)) return fail(EPLL_EINVAL, "blur kernel must have a positive sum");
        } else if (deg->kind != EPLL_DENOISE) {
            return fail(EPLL_EINVAL, "unknown degradation kind");
        }
    }
    return EPLL_OK;
}

}  // namespace epll

using namespace epll;

extern "C" {

const char *epll_last_error(void) { return g_err.c_str(); }

void epll_options_default(epll_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = EPLL_FP32;
    o->tie_gap = -1.0f;
    o->subset = EPLL_SUBSET_ALL;
    o->subset_param = 0.0;
    o->seed = 0;
    o->cg_iters = 100;
    o->select = EPLL_SELECT_EXHAUSTIVE;
}

// tile_pack: lay the components out so that none straddles a 256-column tile
// (the grouping of the tensor-core selection's ragged-rank epilogue); the
// node model of a search tree keeps consecutive children contiguous instead.
static epll_status gmm_load_impl(int K, int P, const double *weights, const double *eigvecs,
                                 const double *eigvals, int rank_mode, double rank_param, bool tile_pack,
                                 epll_gmm **out)
{
    if (!out) return fail(EPLL_EINVAL, "null output handle pointer");
    *out = nullptr;
    if (K < 1 || K > 4096) return fail(EPLL_EINVAL, "K must be in 1..4096");
    if (P != PD) return fail(EPLL_EINVAL, "P must be 64 (8x8 patches)");
    if (!weights || !eigvecs || !eigvals) return fail(EPLL_EINVAL, "null model array");
    if (rank_mode == EPLL_RANK_FIXED) {
        if (!(rank_param >= 1.0 && rank_param <= PD) || rank_param != std::floor(rank_param))
            return fail(EPLL_EINVAL, "fixed rank must be an integer in 1..64");
    } else if (rank_mode == EPLL_RANK_RHO) {
        if (!(rank_param > 0.0 && rank_param <= 1.0)) return fail(EPLL_EINVAL, "rho must be in (0, 1]");
    } else {
        return fail(EPLL_EINVAL, "unknown rank mode");
    }
    double wsum = 0.0;
    for (int k = 0; k < K; ++k) {
        if (!(weights[k] > 0.0) || !std::isfinite(weights[k])) return fail(EPLL_EINVAL, "weights must be positive");
        wsum += weights[k];
        for (int j = 0; j < PD; ++j) {
            double s = eigvals[(size_t)k * PD + j];
            if (!(s > 0.0) || !std::isfinite(s)) return fail(EPLL_EINVAL, "eigenvalues must be positive");
            if (j && s > eigvals[(size_t)k * PD + j - 1]) return fail(EPLL_EINVAL, "eigenvalues must be non-increasing");
        }
    }
    for (size_t q = 0; q < (size_t)K * PD * PD; ++q)
        if (!std::isfinite(eigvecs[q])) return fail(EPLL_EINVAL, "eigenvectors must be finite");

    epll_gmm *g = new epll_gmm();
    g->K = K;
    g->rank_mode = rank_mode;
    g->rank_param = rank_param;
    g->h_r = new int[K];
    g->h_lam = new double[K];
    g->h_roff = new int[K + 1];
    // flat tail (Sec. "Speed-up via flat tail spectrum approximation")
    for (int k = 0; k < K; ++k) {
        const double *s = eigvals + (size_t)k * PD;
        int rk = PD;
        if (rank_mode == EPLL_RANK_FIXED) {
            rk = (int)rank_param;
        } else {
            double tot = 0.0, acc = 0.0;
            for (int j = 0; j < PD; ++j) tot += s[j];
            for (int j = 0; j < PD; ++j) {
                acc += s[j];
                if (acc >= rank_param * tot) { rk = j + 1; break; }
            }
        }
        double tail = 0.0;
        for (int j = rk; j < PD; ++j) tail += s[j];
        g->h_r[k] = rk;
        g->h_lam[k] = rk < PD ? tail / (double)(PD - rk) : 0.0;
    }
    // column layout: component k at h_roff[k], its rank padded to a multiple
    // of 8 columns; with tile_pack a component that would cross a 256-column
    // boundary starts at the next tile (the skipped columns belong to no
    // component)
    std::vector<int> width(K);
    {
        int pos = 0;
        for (int k = 0; k < K; ++k) {
            width[k] = (g->h_r[k] + COL_ALIGN - 1) / COL_ALIGN * COL_ALIGN;
            if (tile_pack && pos % RTOT_ALIGN + width[k] > RTOT_ALIGN)
                pos = (pos + RTOT_ALIGN - 1) / RTOT_ALIGN * RTOT_ALIGN;
            g->h_roff[k] = pos;
            pos += width[k];
        }
        g->h_roff[K] = pos;
    }
    g->Rtot = (g->h_roff[K] + RTOT_ALIGN - 1) / RTOT_ALIGN * RTOT_ALIGN;
    g->rank_sum = 0;
    for (int k = 0; k < K; ++k) g->rank_sum += g->h_r[k];
    g->uniform_rank = g->h_r[0];
    for (int k = 1; k < K; ++k)
        if (g->h_r[k] != g->h_r[0]) g->uniform_rank = 0;
    if (g->uniform_rank != 8 && g->uniform_rank != 16 && g->uniform_rank != 64) g->uniform_rank = 0;
    g->h_roff[K] = g->Rtot;  // trailing padding columns belong to the last component
    const int R = g->Rtot;

    std::vector<double> w(K);
    for (int k = 0; k < K; ++k) w[k] = weights[k] / wsum;
    std::vector<float> B((size_t)PD * R, 0.0f), Blo((size_t)PD * R, 0.0f);
    std::vector<int> colk(R, -1);
    for (int k = 0; k < K; ++k) {
        // the component's padded width; the trailing columns of the last tile
        // belong to the last component (zero basis columns)
        const int cend = k + 1 < K ? g->h_roff[k] + width[k] : R;
        for (int c = g->h_roff[k]; c < cend; ++c) colk[c] = k;
        for (int e = 0; e < PD; ++e)
            for (int j = 0; j < g->h_r[k]; ++j) {
                const double u = eigvecs[((size_t)k * PD + e) * PD + j];
                const float h = (float)u;
                B[(size_t)e * R + g->h_roff[k] + j] = h;
                Blo[(size_t)e * R + g->h_roff[k] + j] = (float)(u - (double)h);
            }
    }
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    // column arrays carry COL_PAD trailing zero entries: a 32-column chunk that
    // starts at an 8-aligned column below Rtot stays inside the allocation
    constexpr int COL_PAD = 64;
    A(dalloc(&g->d_r, K)); A(dalloc(&g->d_roff, K + 1)); A(dalloc(&g->d_colk, R + COL_PAD));
    A(dalloc(&g->d_S, (size_t)K * PD)); A(dalloc(&g->d_w, K)); A(dalloc(&g->d_lam, K));
    A(dalloc(&g->d_B, (size_t)PD * R + COL_PAD)); A(dalloc(&g->d_Blo, (size_t)PD * R + COL_PAD));
    A(dalloc(&g->d_Ub, 2 * (size_t)PD * R)); A(dalloc(&g->d_U2b, 2 * (size_t)PD * R));
    A(dalloc(&g->d_tileg, R / RTOT_ALIGN));
    g->Rp = R + COL_PAD;
    A(alloc_tables(g));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_model(g);
        delete g;
        return fail(EPLL_ENOMEM, std::string("model allocation: ") + cudaGetErrorString(e));
    }
    A(cudaMemcpy(g->d_r, g->h_r, sizeof(int) * K, cudaMemcpyHostToDevice));
    A(cudaMemcpy(g->d_roff, g->h_roff, sizeof(int) * (K + 1), cudaMemcpyHostToDevice));
    A(cudaMemset(g->d_colk, 0, sizeof(int) * (R + COL_PAD)));
    A(cudaMemset(g->d_B, 0, sizeof(float) * ((size_t)PD * R + COL_PAD)));
    A(cudaMemset(g->d_Blo, 0, sizeof(float) * ((size_t)PD * R + COL_PAD)));
    A(cudaMemcpy(g->d_colk, colk.data(), sizeof(int) * R, cudaMemcpyHostToDevice));
    {
        // the four epilogue column groups of every 256-column tile: group h
        // starts at the first component starting at or after column 64 h of
        // the tile (the tile's end when there is none); components never
        // straddle a group when the layout is tile-packed
        const int nt = R / RTOT_ALIGN;
        std::vector<int4> tg(nt);
        for (int t = 0; t < nt; ++t) {
            int b[4] = {0, RTOT_ALIGN, RTOT_ALIGN, RTOT_ALIGN};
            for (int h = 1; h < 4; ++h)
                for (int k = 0; k < K; ++k) {
                    const int rel = g->h_roff[k] - t * RTOT_ALIGN;
                    if (rel >= 64 * h && rel < RTOT_ALIGN) {
                        b[h] = rel;
                        break;
                    }
                }
            for (int h = 2; h < 4; ++h) b[h] = std::max(b[h], b[h - 1]);
            tg[t] = make_int4(b[0], b[1], b[2], b[3]);
        }
        A(cudaMemcpy(g->d_tileg, tg.data(), sizeof(int4) * nt, cudaMemcpyHostToDevice));
    }
    A(cudaMemcpy(g->d_S, eigvals, sizeof(double) * K * PD, cudaMemcpyHostToDevice));
    A(cudaMemcpy(g->d_w, w.data(), sizeof(double) * K, cudaMemcpyHostToDevice));
    A(cudaMemcpy(g->d_lam, g->h_lam, sizeof(double) * K, cudaMemcpyHostToDevice));
    A(cudaMemcpy(g->d_B, B.data(), sizeof(float) * B.size(), cudaMemcpyHostToDevice));
    A(cudaMemcpy(g->d_Blo, Blo.data(), sizeof(float) * Blo.size(), cudaMemcpyHostToDevice));
    {
        // split BF16 copies of B (hi = BF16(b), lo = BF16(b - hi)) in both
        // orientations for the tensor-core estimation
        const size_t PR = (size_t)PD * R;
        std::vector<uint16_t> ub(2 * PR), u2b(2 * PR);
        for (int ee = 0; ee < PD; ++ee)
            for (int j = 0; j < R; ++j) {
                const float b = B[(size_t)ee * R + j];
                const uint16_t h = bf16_bits(b), l = bf16_bits(b - bf16_value(h));
                ub[(size_t)j * PD + ee] = h;
                ub[PR + (size_t)j * PD + ee] = l;
                u2b[(size_t)ee * R + j] = h;
                u2b[PR + (size_t)ee * R + j] = l;
            }
        A(cudaMemcpy(g->d_Ub, ub.data(), sizeof(uint16_t) * ub.size(), cudaMemcpyHostToDevice));
        A(cudaMemcpy(g->d_U2b, u2b.data(), sizeof(uint16_t) * u2b.size(), cudaMemcpyHostToDevice));
    }
    if (e != cudaSuccess) {
        free_model(g);
        delete g;
        return fail(EPLL_ECUDA, std::string("model upload: ") + cudaGetErrorString(e));
    }
    cg_setup();
    group_setup();
    sampler_setup();
    *out = g;
    return EPLL_OK;
}

void epll_gmm_free(epll_gmm *g)
{
    if (!g) return;
    cudaDeviceSynchronize();
    if (g->aux) cudaStreamDestroy(g->aux);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    free_workspace(g->ws);
    free_model(g);
    delete g;
}

epll_status epll_gmm_load(int K, int P, const double *weights, const double *eigvecs,
                          const double *eigvals, int rank_mode, double rank_param, epll_gmm **out)
{
    return gmm_load_impl(K, P, weights, eigvecs, eigvals, rank_mode, rank_param, true, out);
}

epll_status epll_gmm_attach_tree(epll_gmm *g, int n_nodes, const double *weights, const double *eigvecs,
                                 const double *eigvals, const int *child_begin, const int *leaf_component)
{
    if (!g || g->lane) return fail(EPLL_EINVAL, "null model handle");
    if (n_nodes == 0) {
        EPLL_CU(cudaDeviceSynchronize());
        free_batch(g);
        free_tree(g);
        return EPLL_OK;
    }
    if (n_nodes < 2 || n_nodes > 65536) return fail(EPLL_EINVAL, "n_nodes must be in 2..65536 (0 detaches)");
    if (!weights || !eigvecs || !eigvals || !child_begin || !leaf_component)
        return fail(EPLL_EINVAL, "null tree array");
    if (child_begin[0] != 1 || child_begin[n_nodes] != n_nodes)
        return fail(EPLL_EINVAL, "child_begin must start at 1 (the root's children) and end at n_nodes");
    std::vector<int> parent(n_nodes, -1), depth(n_nodes, 0);
    std::vector<char> seen(g->K, 0);
    int leaves = 0, leaf_depth = -1;
    for (int v = 0; v < n_nodes; ++v) {
        const int b = child_begin[v], e = child_begin[v + 1];
        if (e < b) return fail(EPLL_EINVAL, "child_begin must be non-decreasing");
        if (e > b) {
            if (b <= v) return fail(EPLL_EINVAL, "nodes must be in breadth-first order (children after their parent)");
            if (e - b > 4) return fail(EPLL_EINVAL, "a node has more than 4 children");
            if (leaf_component[v] != -1) return fail(EPLL_EINVAL, "an internal node has a leaf component");
            for (int c = b; c < e; ++c) parent[c] = v;
        } else {
            const int k = leaf_component[v];
            if (k < 0 || k >= g->K || seen[k]) return fail(EPLL_EINVAL, "leaves must map to distinct components");
            seen[k] = 1;
            ++leaves;
        }
    }
    if (leaves != g->K) return fail(EPLL_EINVAL, "every component must be a leaf");
    for (int v = 1; v < n_nodes; ++v) depth[v] = depth[parent[v]] + 1;
    for (int v = 0; v < n_nodes; ++v)
        if (child_begin[v] == child_begin[v + 1]) {
            if (leaf_depth < 0) leaf_depth = depth[v];
            if (depth[v] != leaf_depth) return fail(EPLL_EINVAL, "every leaf must be at the same depth");
        }
    if (leaf_depth < 1 || leaf_depth > 32) return fail(EPLL_EINVAL, "tree depth must be in 1..32");
    epll_gmm *tm = nullptr;
    epll_status s = gmm_load_impl(n_nodes, PD, weights, eigvecs, eigvals, g->rank_mode, g->rank_param, false, &tm);
    if (s) return s;
    double cols = 0.0;
    int internal = 0;
    for (int v = 0; v < n_nodes; ++v)
        if (child_begin[v + 1] > child_begin[v]) {
            const int last = child_begin[v + 1] - 1;
            const int c = tm->h_roff[last] + (tm->h_r[last] + COL_ALIGN - 1) / COL_ALIGN * COL_ALIGN -
                          tm->h_roff[child_begin[v]];
            if (c > 256) {
                epll_gmm_free(tm);
                return fail(EPLL_EINVAL, "a node's children have more than 256 basis columns");
            }
            cols += c;
            ++internal;
        }
    TreeState *tr = new TreeState();
    tr->tm = tm;
    tr->n_nodes = n_nodes;
    tr->depth = leaf_depth;
    tr->child_cols_mean = cols / internal;
    cudaError_t e = cudaMalloc(&tr->d_child, sizeof(int) * (n_nodes + 1));
    if (e == cudaSuccess) e = cudaMalloc(&tr->d_leaf, sizeof(int) * n_nodes);
    if (e == cudaSuccess) e = cudaMemcpy(tr->d_child, child_begin, sizeof(int) * (n_nodes + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(tr->d_leaf, leaf_component, sizeof(int) * n_nodes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        epll_gmm tmp;
        tmp.tree = tr;
        free_tree(&tmp);
        return fail(EPLL_ENOMEM, std::string("tree upload: ") + cudaGetErrorString(e));
    }
    EPLL_CU(cudaDeviceSynchronize());
    free_batch(g);
    free_tree(g);
    g->tree = tr;
    return EPLL_OK;
}

epll_status epll_gmm_ranks(const epll_gmm *g, int *ranks, double *lambdas)
{
    if (!g) return fail(EPLL_EINVAL, "null model handle");
    if (ranks) std::memcpy(ranks, g->h_r, sizeof(int) * g->K);
    if (lambdas) std::memcpy(lambdas, g->h_lam, sizeof(double) * g->K);
    return EPLL_OK;
}

epll_status epll_restore(epll_gmm *g, const float *y, int H, int W, const epll_degradation *deg,
                         float sigma, const double *beta_mult, int T, const epll_options *opt,
                         float *x_out, void *stream)
{
    epll_options o;
    if (opt) o = *opt; else epll_options_default(&o);
    epll_status s;
    if ((s = check_restore_args(g, y, H, W, deg, sigma, beta_mult, T, o, x_out))) return s;
    if ((s = ensure_workspace(g, (size_t)H * W))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const float *a = (deg && deg->kind == EPLL_PIXELWISE) ? deg->a : nullptr;
    if ((s = run_restore(g, y, a, H, W, deg, sigma, beta_mult, T, o, st))) return s;
    EPLL_CU(cudaMemcpyAsync(x_out, g->ws.xhat, sizeof(float) * (size_t)H * W, cudaMemcpyDeviceToDevice, st));
    return EPLL_OK;
}

epll_status epll_restore_host(epll_gmm *g, const float *y, int H, int W, const epll_degradation *deg,
                              float sigma, const double *beta_mult, int T, const epll_options *opt,
                              float *x_out, void *stream)
{
    epll_options o;
    if (opt) o = *opt; else epll_options_default(&o);
    epll_status s;
    if ((s = check_restore_args(g, y, H, W, deg, sigma, beta_mult, T, o, x_out))) return s;
    if ((s = ensure_workspace(g, (size_t)H * W))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace &ws = g->ws;
    const size_t bytes = sizeof(float) * (size_t)H * W;
    const size_t dd = (deg && deg->kind == EPLL_CONV_DECIMATE) ? (size_t)deg->factor * deg->factor : 1;
    EPLL_CU(cudaMemcpyAsync(ws.y, y, bytes / dd, cudaMemcpyHostToDevice, st));
    const float *a = nullptr;
    if (deg && deg->kind == EPLL_PIXELWISE) {
        EPLL_CU(cudaMemcpyAsync(ws.a, deg->a, bytes, cudaMemcpyHostToDevice, st));
        a = ws.a;
    }
    if ((s = run_restore(g, ws.y, a, H, W, deg, sigma, beta_mult, T, o, st))) return s;
    EPLL_CU(cudaMemcpyAsync(x_out, ws.xhat, bytes, cudaMemcpyDeviceToHost, st));
    EPLL_CU(cudaStreamSynchronize(st));
    return EPLL_OK;
}

epll_status epll_image_update(epll_gmm *g, const float *y, const float *xtilde, int H, int W,
                              const epll_degradation *deg, float sigma, double beta_mult, float *x_out,
                              void *stream)
{
    if (!g) return fail(EPLL_EINVAL, "null model handle");
    if (!xtilde) return fail(EPLL_EINVAL, "null image pointer");
    if (!(beta_mult > 0.0) || !std::isfinite(beta_mult)) return fail(EPLL_EINVAL, "beta multiplier must be positive");
    epll_options o;
    epll_options_default(&o);
    epll_status s;
    if ((s = check_restore_args(g, y, H, W, deg, sigma, nullptr, 0, o, x_out))) return s;
    if ((s = ensure_workspace(g, (size_t)H * W))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace &ws = g->ws;
    const int kind = deg ? deg->kind : EPLL_DENOISE;
    const float *a = kind == EPLL_PIXELWISE ? deg->a : nullptr;
    g->launches = 0;
    if (kind == EPLL_CONV_PERIODIC || kind == EPLL_CONV_DECIMATE) {
        const int d = kind == EPLL_CONV_DECIMATE ? deg->factor : 1;
        if (kind == EPLL_CONV_PERIODIC) {
            if ((s = fft_prepare(g, deg->kernel, deg->kh, deg->kw, y, H, W, st))) return s;
        } else {
            if ((s = sr_prepare(g, deg->kernel, deg->kh, deg->kw, y, H, W, d, st))) return s;
        }
        if ((s = launch_lambda(g, kind, a, H, W, sigma, st, d))) return s;
        EPLL_CU(cudaMemcpyAsync(ws.xtil, xtilde, sizeof(float) * (size_t)H * W, cudaMemcpyDeviceToDevice, st));
        if (kind == EPLL_CONV_PERIODIC) {
            if ((s = fft_update(g, H, W, beta_mult, st))) return s;
        } else {
            if ((s = sr_update(g, H, W, d, beta_mult, st))) return s;
        }
        EPLL_CU(cudaMemcpyAsync(x_out, ws.xhat, sizeof(float) * (size_t)H * W, cudaMemcpyDeviceToDevice, st));
    } else {
        if ((s = launch_lambda(g, kind, a, H, W, sigma, st))) return s;
        if ((s = launch_pixel_update(g, a, y, xtilde, H, W, beta_mult, x_out, st))) return s;
    }
    g->last_launches = g->launches;
    return EPLL_OK;
}

__global__ void k_iota(int *out, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = i;
}

epll_status epll_patch_step(epll_gmm *g, const float *xhat, int H, int W, double beta,
                            const epll_options *opt, int t, float *xtilde, int *anchors,
                            int *kstar, float *gap, const int *forced_k, int *n_out, void *stream)
{
    if (!g) return fail(EPLL_EINVAL, "null model handle");
    if (!xhat || !xtilde) return fail(EPLL_EINVAL, "null image pointer");
    if (!(beta > 0.0) || !std::isfinite(beta)) return fail(EPLL_EINVAL, "beta must be positive");
    epll_options o;
    if (opt) o = *opt; else epll_options_default(&o);
    epll_status s;
    if ((s = check_image(H, W))) return s;
    if ((s = check_options(o, H, W))) return s;
    if ((s = check_select(g, o))) return s;
    if ((s = ensure_workspace(g, (size_t)H * W))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace &ws = g->ws;
    g->launches = 0;
    g->last_evals = 0;
    EPLL_CU(cudaMemsetAsync(ws.ctr, 0, sizeof(long long) * 4, st));
    EPLL_CU(cudaMemsetAsync(cnt(g, CNT_ERR), 0, sizeof(int), st));
    int n = 0;
    const double one = 1.0;
    if ((s = prepare_batch(g, H, W, o, t, 1, ws.scal, &one, 1.0, beta, &n, st))) return s;
    use_slot(g, 0, (size_t)H * W);
    if ((s = patch_phase(g, xhat, H, W, o, n, forced_k, st))) return s;
    const unsigned *mult = o.subset == EPLL_SUBSET_ALL ? nullptr : ws.mult;
    if ((s = launch_aggregate(g, xhat, H, W, mult, nullptr, nullptr, ws.lamf, 0.0, xtilde, st))) return s;
    if (anchors) {
        if (o.subset == EPLL_SUBSET_ALL) {
            k_iota<<<(n + 255) / 256, 256, 0, st>>>(anchors, n);
            EPLL_LAUNCHED(g);
        } else {
            EPLL_CU(cudaMemcpyAsync(anchors, ws.anchors, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st));
        }
    }
    if (kstar) EPLL_CU(cudaMemcpyAsync(kstar, ws.kstar, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    if (gap) EPLL_CU(cudaMemcpyAsync(gap, ws.gap, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    g->last_launches = g->launches;
    if (n_out) {
        EPLL_CU(cudaStreamSynchronize(st));
        int timed_out = 0;
        EPLL_CU(cudaMemcpy(&timed_out, cnt(g, CNT_ERR), sizeof(int), cudaMemcpyDeviceToHost));
        if (timed_out) return fail(EPLL_ETIMEOUT, "a tensor-core selection kernel gave up on a bounded wait");
        *n_out = n;
    }
    return EPLL_OK;
}

epll_status epll_sample(int H, int W, const epll_options *opt, int t, int *anchors, int *n_out,
                        void *stream)
{
    if (!anchors || !n_out) return fail(EPLL_EINVAL, "null output pointer");
    epll_options o;
    if (opt) o = *opt; else epll_options_default(&o);
    epll_status s;
    if ((s = check_image(H, W))) return s;
    if ((s = check_options(o, H, W))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)H * W;
    epll_gmm tmp;
    unsigned *mult = nullptr;
    const size_t sstride = sampler_stride(N);
    if (dalloc(&tmp.ws.sampler, sstride) != cudaSuccess || dalloc(&mult, N) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(tmp.ws.sampler);
        cudaFree(mult);
        return fail(EPLL_ENOMEM, "sampler scratch allocation failed");
    }
    int n = 0;
    s = launch_sample(&tmp, H, W, o, t, 1, &n, anchors, mult, tmp.ws.sampler, sstride, st);
    if (s == EPLL_OK && o.subset == EPLL_SUBSET_ALL) {
        k_iota<<<(n + 255) / 256, 256, 0, st>>>(anchors, n);
        if (cudaGetLastError() != cudaSuccess) s = fail(EPLL_ECUDA, "iota launch failed");
    }
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(tmp.ws.sampler);
    cudaFree(mult);
    tmp.ws.sampler = nullptr;
    if (s) return s;
    if (e != cudaSuccess) return fail(EPLL_ECUDA, std::string("sampler: ") + cudaGetErrorString(e));
    *n_out = n;
    return EPLL_OK;
}

epll_status epll_profile_enable(epll_gmm *g, int enable)
{
    if (!g) return fail(EPLL_EINVAL, "null model handle");
    if (enable && !g->prof_ev) {
        g->prof_ev = new cudaEvent_t[2 * PROF_MAX];
        for (int i = 0; i < 2 * PROF_MAX; ++i) EPLL_CU(cudaEventCreate(&g->prof_ev[i]));
    }
    g->prof_on = enable != 0;
    return EPLL_OK;
}

epll_status epll_profile_read(epll_gmm *g, double *ms, long long *launches, double *flops)
{
    if (!g) return fail(EPLL_EINVAL, "null model handle");
    EPLL_CU(cudaDeviceSynchronize());
    double tot = 0.0;
    for (int i = 0; i < g->prof_n; ++i) {
        float t = 0.0f;
        EPLL_CU(cudaEventElapsedTime(&t, g->prof_ev[2 * i], g->prof_ev[2 * i + 1]));
        tot += t;
    }
    if (ms) *ms = tot;
    if (launches) *launches = g->prof_n;
    if (flops) *flops = g->prof_flops;
    g->prof_n = 0;
    g->prof_flops = 0.0;
    return EPLL_OK;
}

epll_status epll_last_counters(epll_gmm *g, long long *patch_evals, long long *rescored,
                               long long *launches)
{
    if (!g) return fail(EPLL_EINVAL, "null model handle");
    EPLL_CU(cudaDeviceSynchronize());
    long long c[4] = {0, 0, 0, 0};
    int timed_out = 0;
    if (g->ws.ctr) EPLL_CU(cudaMemcpy(c, g->ws.ctr, sizeof(c), cudaMemcpyDeviceToHost));
    if (g->ws.counts)
        EPLL_CU(cudaMemcpy(&timed_out, cnt(g, CNT_ERR), sizeof(int), cudaMemcpyDeviceToHost));
    if (patch_evals) *patch_evals = g->last_evals;
    if (rescored) *rescored = c[0];
    if (launches) *launches = g->last_launches;
    if (timed_out) return fail(EPLL_ETIMEOUT, "a tensor-core selection kernel gave up on a bounded wait");
    return EPLL_OK;
}

epll_status epll_last_fallbacks(epll_gmm *g, long long *fallbacks)
{
    if (!g || !fallbacks) return fail(EPLL_EINVAL, "null argument");
    EPLL_CU(cudaDeviceSynchronize());
    long long c[4] = {0, 0, 0, 0};
    if (g->ws.ctr) EPLL_CU(cudaMemcpy(c, g->ws.ctr, sizeof(c), cudaMemcpyDeviceToHost));
    *fallbacks = c[1];
    return EPLL_OK;
}

}  // extern "C"
