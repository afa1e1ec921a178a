// Patch-step kernels of Algorithm 1: patch extraction, Gaussian selection
// (FP32 SIMT form), near-tie rescoring in compensated FP32, grouping of the
// patches by selected component, Wiener patch estimation (Eqs. 15-16) and
// patch reprojection by overlap-add averaging fused with the image update.
#include "epll_internal.cuh"

#include <cooperative_groups.h>

#include <cfloat>
#include <climits>

namespace epll {

// Periodic 8x8 patch at anchor a (top-left pixel), element e = 8u + v.
__device__ __forceinline__ size_t pix(int ai, int aj, int u, int v, int H, int W)
{
    int i = ai + u;
    if (i >= H) i -= H;
    int j = aj + v;
    if (j >= W) j -= W;
    return (size_t)i * W + j;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ============================================================================
// Gaussian selection, FP32 SIMT form.  One thread per sampled patch: the
// thread extracts its DC-free patch into registers, then streams the
// concatenated bases [Ubar_1 ... Ubar_K] (64 x Rtot) through shared memory in
// chunks of SEL_CH columns, forming c = Ubar^T z (Eq. 13) and the score of
// Eq. 14 component by component, keeping the best and second-best score.
// Patches whose top-2 gap is below tau are appended to the near-tie list.
// ============================================================================
constexpr int SEL_THREADS = 128;
constexpr int SEL_CH = 32;

// DUMP = true: the patches are entries [f0, f0 + fcap) of a device list (count
// *nlist) and every component's score is written to scores[(f - f0) * K + k].
// In list mode blockIdx.y selects a slice of whole components (columns
// [roff[k0], roff[k1])) so that a short list still spreads over many blocks.
template <bool DUMP>
__global__ void __launch_bounds__(SEL_THREADS)
k_select_fp32(const float *__restrict__ xhat, int H, int W, const int *__restrict__ anchors, int n,
              const float *__restrict__ B, int Rtot, const int *__restrict__ colk, Tables tab,
              float tau_abs, float tau_rel, int *__restrict__ kstar, float *__restrict__ gap,
              int *__restrict__ flag, int *__restrict__ nflag, const int *__restrict__ list,
              const int *__restrict__ nlist, int f0, int fcap, int K, const int *__restrict__ roff,
              float *__restrict__ scores)
{
    pdl_enter();
    __shared__ __align__(16) float Bs[PD][SEL_CH];
    __shared__ float qs[SEL_CH];
    __shared__ int ks[SEL_CH];
    int i = blockIdx.x * SEL_THREADS + threadIdx.x;
    bool valid = i < n;
    int f = 0, cbeg = 0, cend = Rtot;
    if (DUMP) {
        const int count = min(*nlist - f0, fcap);
        if ((int)(blockIdx.x * SEL_THREADS) >= count) return;  // whole block idle
        f = i;
        valid = f < count;
        i = valid ? list[f0 + f] : 0;
        const int k0 = (int)((long long)K * blockIdx.y / gridDim.y);
        const int k1 = (int)((long long)K * (blockIdx.y + 1) / gridDim.y);
        if (k0 == k1) return;
        cbeg = roff[k0];
        cend = roff[k1];
    }

    float z[PD];
    float zz = 0.0f;
    {
        const int a = valid ? (anchors ? anchors[i] : i) : 0;
        const int ai = a / W, aj = a % W;
        float m = 0.0f;
#pragma unroll
        for (int u = 0; u < PS; ++u)
#pragma unroll
            for (int v = 0; v < PS; ++v) {
                z[u * PS + v] = xhat[pix(ai, aj, u, v, H, W)];
                m += z[u * PS + v];
            }
        m *= (1.0f / PD);
#pragma unroll
        for (int e = 0; e < PD; ++e) {
            z[e] -= m;
            zz = fmaf(z[e], z[e], zz);
        }
    }

    float s1 = FLT_MAX, s2 = FLT_MAX, acc = 0.0f;
    int k1 = 0, curk = -1;
    for (int c0 = cbeg; c0 < cend; c0 += SEL_CH) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < PD * SEL_CH / 4; idx += SEL_THREADS) {
            const int e = idx / (SEL_CH / 4), c4 = idx % (SEL_CH / 4);
            reinterpret_cast<float4 *>(&Bs[e][0])[c4] =
                *reinterpret_cast<const float4 *>(B + (size_t)e * Rtot + c0 + 4 * c4);
        }
        if (threadIdx.x < SEL_CH) {
            qs[threadIdx.x] = tab.q_hi[c0 + threadIdx.x];
            ks[threadIdx.x] = colk[c0 + threadIdx.x];
        }
        __syncthreads();
        float c[SEL_CH];
#pragma unroll
        for (int cc = 0; cc < SEL_CH; ++cc) c[cc] = 0.0f;
#pragma unroll
        for (int e = 0; e < PD; ++e) {
            const float ze = z[e];
#pragma unroll
            for (int c4 = 0; c4 < SEL_CH / 4; ++c4) {
                const float4 b = reinterpret_cast<const float4 *>(&Bs[e][0])[c4];
                c[4 * c4 + 0] = fmaf(ze, b.x, c[4 * c4 + 0]);
                c[4 * c4 + 1] = fmaf(ze, b.y, c[4 * c4 + 1]);
                c[4 * c4 + 2] = fmaf(ze, b.z, c[4 * c4 + 2]);
                c[4 * c4 + 3] = fmaf(ze, b.w, c[4 * c4 + 3]);
            }
        }
#pragma unroll
        for (int cc = 0; cc < SEL_CH; ++cc) {
            if (DUMP && c0 + cc >= cend) break;  // slice ends inside the chunk (uniform)
            const int k = ks[cc];
            if (k != curk) {
                if (curk >= 0) {
                    const float s = tab.cst_hi[curk] + tab.t_hi[curk] * zz + acc;
                    if (DUMP) {
                        if (valid) scores[(size_t)f * K + curk] = s;
                    } else if (s < s1) { s2 = s1; s1 = s; k1 = curk; }
                    else if (s < s2) { s2 = s; }
                }
                curk = k;
                acc = 0.0f;
            }
            acc = fmaf(qs[cc] * c[cc], c[cc], acc);
        }
    }
    {
        const float s = tab.cst_hi[curk] + tab.t_hi[curk] * zz + acc;
        if (DUMP) {
            if (valid) scores[(size_t)f * K + curk] = s;
            return;
        }
        if (s < s1) { s2 = s1; s1 = s; k1 = curk; }
        else if (s < s2) { s2 = s; }
    }
    if (valid) {
        kstar[i] = k1;
        const float gp = s2 - s1;
        gap[i] = gp;
        if (!(gp >= tau_abs + tau_rel * zz * tab.tmax[0])) flag[atomicAdd(nflag, 1)] = i;
    }
}

epll_status launch_select_fp32(epll_gmm *g, const float *xhat, int H, int W, const int *anchors,
                               int n, float tau_abs, float tau_rel, cudaStream_t st)
{
    Workspace &ws = g->ws;
    int *nflag = cnt(g, CNT_NFLAG);
    EPLL_CU(cudaMemsetAsync(nflag, 0, sizeof(int), st));
    prof_begin(g, st);
    EPLL_CU(launch_pdl(k_select_fp32<false>, dim3((n + SEL_THREADS - 1) / SEL_THREADS), dim3(SEL_THREADS), 0, st, 
        xhat, H, W, anchors, n, g->d_B, g->Rtot, g->d_colk, g->tab, tau_abs, tau_rel, ws.kstar, ws.gap,
        ws.flag, nflag, nullptr, nullptr, 0, 0, g->K, g->d_roff, nullptr));
    prof_end(g, st, n);
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

// ============================================================================
// Near-tie rescoring.  The FP32 kernel above, in list mode, first writes all
// K scores of every listed patch (block-tiled, the bases streamed through
// shared memory).  Then one warp per listed patch rescores, in compensated
// arithmetic, every component within the FP32 error band of the best: the
// patch, its mean, the basis (float value + float rounding error of the FP64
// eigenvectors) and the FP64 tables are carried as unevaluated sums of two
// floats (Dekker's TwoSum / TwoProduct with FMA), which resolves the
// selection like FP64 arithmetic would.  The winner and its gap overwrite
// kstar / gap.
// ============================================================================
struct df {
    float hi, lo;
};
__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    float s = a + b;
    float e = b - (s - a);
    return {s, e};
}
__device__ __forceinline__ df df_add(df x, df y)
{
    df s = two_sum(x.hi, y.hi);
    df t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df x, df y)
{
    float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_shfl_xor(df v, int o)
{
    return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ df df_warp_sum(df v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
    return v;
}
// x < y for unevaluated sums
__device__ __forceinline__ bool df_less(df x, df y)
{
    df d = df_add(x, {-y.hi, -y.lo});
    return d.hi < 0.0f || (d.hi == 0.0f && d.lo < 0.0f);
}

// FP32 pass-1 band: absolute + relative to |z|^2 max 1/nu (the FP32 error scale)
constexpr float RESCORE_ABS = 1e-3f;
constexpr float RESCORE_REL = 2e-5f;
constexpr int RS_WARPS = 8;
constexpr int RS_QW = 4;                  // warps per candidate: each sums 16 of the 64 terms
constexpr int RS_CPR = RS_WARPS / RS_QW;  // candidates per round
constexpr int RS_KMAX = 4096;             // candidate list capacity (the model's K at most)

// Entries [f0, f0 + fcap) of the near-tie list; scores[(f - f0) * K + k] holds
// each component's dumped score.  A block takes one listed patch: warp 0
// forms the compensated DC-free patch and |z|^2 while the block finds the
// best dumped score and lists the components within the band of it (all
// their loads issued at once).  The candidates are then rescored two at a
// time, four warps each: warp quarter qq forms, for coefficients j = lane
// and lane + 32, the compensated partial sum of c_j = u_j . z over the terms
// 16 qq .. 16 qq + 15 (its 64 basis loads independent of each other); the
// candidate's first warp adds the four partials in order and forms the
// score.  The best and second best (compensated; the lower component on
// equal scores) are merged at the end.
__global__ void __launch_bounds__(32 * RS_WARPS)
k_rescore(const float *__restrict__ xhat, int H, int W, const int *__restrict__ anchors,
          const int *__restrict__ flag, const int *__restrict__ nflag, int f0, int fcap, int K,
          int Rtot, const int *__restrict__ roff, const int *__restrict__ rk_,
          const float *__restrict__ B, const float *__restrict__ Blo, Tables tab,
          const float *__restrict__ scores, float band_abs, float band_rel, int *__restrict__ kstar,
          float *__restrict__ gap, long long *__restrict__ ctr)
{
    pdl_enter();
    __shared__ float zh[PD], zl[PD];
    __shared__ df s_zz;
    __shared__ float s_red[RS_WARPS];
    __shared__ int s_cand[RS_KMAX];
    __shared__ int s_cor[RS_KMAX];  // the candidate's column offset << 7 | its rank
    __shared__ int s_nc;
    __shared__ df s_part[RS_CPR][RS_QW][PD];
    __shared__ df r_b1[RS_WARPS], r_b2[RS_WARPS];
    __shared__ int r_kb[RS_WARPS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = min(*nflag - f0, fcap);
    if (blockIdx.x == 0 && threadIdx.x == 0 && total > 0)
        atomicAdd((unsigned long long *)ctr, (unsigned long long)total);
    for (int f = blockIdx.x; f < total; f += gridDim.x) {
        const int i = flag[f0 + f];
        const float *sc = scores + (size_t)f * K;
        if (w == 0) {
            const int a = anchors ? anchors[i] : i;
            const int ai = a / W, aj = a % W;
            const float x0 = xhat[pix(ai, aj, lane >> 3, lane & 7, H, W)];
            const float x1 = xhat[pix(ai, aj, (lane >> 3) + 4, lane & 7, H, W)];
            // mean and DC-free patch, compensated
            df sx = df_warp_sum(two_sum(x0, x1));
            df mu = {sx.hi * (1.0f / PD), sx.lo * (1.0f / PD)};
            df z0 = df_add({x0, 0.0f}, {-mu.hi, -mu.lo});
            df z1 = df_add({x1, 0.0f}, {-mu.hi, -mu.lo});
            df zz = df_warp_sum(df_add(df_mul(z0, z0), df_mul(z1, z1)));
            zh[lane] = z0.hi; zl[lane] = z0.lo;
            zh[lane + 32] = z1.hi; zl[lane + 32] = z1.lo;
            if (lane == 0) {
                s_zz = zz;
                s_nc = 0;
            }
        }
        // best dumped score (block-wide)
        float best = FLT_MAX;
        for (int k = threadIdx.x; k < K; k += 32 * RS_WARPS) best = fminf(best, sc[k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0) s_red[w] = best;
        __syncthreads();
        best = s_red[0];
#pragma unroll
        for (int q = 1; q < RS_WARPS; ++q) best = fminf(best, s_red[q]);
        const df zz = s_zz;
        const float band = band_abs + band_rel * (zz.hi + zz.lo) * tab.tmax[0];
        // the components within the band (any order: the merge is order-free)
        float outside = FLT_MAX;
        for (int k = threadIdx.x; k < K; k += 32 * RS_WARPS) {
            const float sk = sc[k];
            if (!(sk > best + band)) {
                const int idx = atomicAdd(&s_nc, 1);
                s_cand[idx] = k;
                s_cor[idx] = (roff[k] << 7) | rk_[k];
            } else {
                outside = fminf(outside, sk);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) outside = fminf(outside, __shfl_xor_sync(0xffffffffu, outside, o));
        __syncthreads();  // s_red is rewritten below; s_cand / s_nc complete
        if (lane == 0) s_red[w] = outside;
        const int nc = s_nc;
        const int slot = w / RS_QW, qq = w % RS_QW;
        df b1 = {FLT_MAX, 0.0f}, b2 = {FLT_MAX, 0.0f};
        int kb = -1;
        for (int c0 = 0; c0 < nc; c0 += RS_CPR) {
            const int ci = c0 + slot;
            const bool mine = ci < nc;  // warp-uniform
            int k = 0, o = 0, r = 0;
            df q0 = {0.0f, 0.0f}, q1 = {0.0f, 0.0f}, tk = {0.0f, 0.0f}, ck = {0.0f, 0.0f};
            if (mine) {
                k = s_cand[ci];
                o = s_cor[ci] >> 7;
                r = s_cor[ci] & 127;
                if (qq == 0) {
                    // the scalars of the score, loaded beside the basis
                    if (lane < r) q0 = {tab.q_hi[o + lane], tab.q_lo[o + lane]};
                    if (lane + 32 < r) q1 = {tab.q_hi[o + lane + 32], tab.q_lo[o + lane + 32]};
                    tk = {tab.t_hi[k], tab.t_lo[k]};
                    ck = {tab.cst_hi[k], tab.cst_lo[k]};
                }
                const int j0 = lane, j1 = lane + 32;
                const float *b0 = B + o + j0, *bl0 = Blo + o + j0;
                df c0s = {0.0f, 0.0f}, c1s = {0.0f, 0.0f};
#pragma unroll
                for (int e = 16 * qq; e < 16 * qq + 16; ++e) {
                    const size_t off = (size_t)e * Rtot;
                    const df z = {zh[e], zl[e]};
                    const df u0 = j0 < r ? df{b0[off], bl0[off]} : df{0.0f, 0.0f};
                    const df u1 = j1 < r ? df{b0[off + 32], bl0[off + 32]} : df{0.0f, 0.0f};
                    c0s = df_add(c0s, df_mul(u0, z));
                    c1s = df_add(c1s, df_mul(u1, z));
                }
                s_part[slot][qq][j0] = c0s;
                s_part[slot][qq][j1] = c1s;
            }
            __syncthreads();
            if (mine && qq == 0) {
                df part = {0.0f, 0.0f};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = lane + 32 * h;
                    if (j < r) {
                        df c = s_part[slot][0][j];
                        c = df_add(c, s_part[slot][1][j]);
                        c = df_add(c, s_part[slot][2][j]);
                        c = df_add(c, s_part[slot][3][j]);
                        part = df_add(part, df_mul(h ? q1 : q0, df_mul(c, c)));
                    }
                }
                df sv = df_warp_sum(part);
                sv = df_add(sv, df_mul(tk, zz));
                sv = df_add(sv, ck);
                if (df_less(sv, b1) || (!df_less(b1, sv) && kb >= 0 && k < kb)) {
                    b2 = b1; b1 = sv; kb = k;
                } else if (df_less(sv, b2)) {
                    b2 = sv;
                }
            }
            __syncthreads();  // s_part is rewritten by the next round
        }
        if (lane == 0) {
            r_b1[w] = b1;
            r_b2[w] = b2;
            r_kb[w] = kb;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            df m1 = {FLT_MAX, 0.0f}, m2 = {FLT_MAX, 0.0f};
            int mk = -1;
            for (int q = 0; q < RS_WARPS; ++q) {
                if (r_kb[q] < 0) continue;
                // merge warp q's best and second best (its best carries r_kb[q])
                const bool first = df_less(r_b1[q], m1) || (!df_less(m1, r_b1[q]) && mk >= 0 && r_kb[q] < mk);
                if (first) {
                    m2 = df_less(r_b2[q], m1) ? r_b2[q] : m1;
                    m1 = r_b1[q];
                    mk = r_kb[q];
                } else {
                    if (df_less(r_b1[q], m2)) m2 = r_b1[q];
                }
            }
            if (mk >= 0) {  // mk < 0 only if every score was NaN
                kstar[i] = mk;
                float out = s_red[0];
                for (int q = 1; q < RS_WARPS; ++q) out = fminf(out, s_red[q]);
                float g2 = (m2.hi == FLT_MAX) ? out - (m1.hi + m1.lo) : (m2.hi - m1.hi) + (m2.lo - m1.lo);
                gap[i] = fminf(g2, out - (m1.hi + m1.lo));
            }
        }
        __syncthreads();
    }
}

epll_status launch_rescore(epll_gmm *g, const float *xhat, int H, int W, const int *anchors,
                           int n, bool split_scores, float tau_abs, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int fcap = (int)ws.fcap;
    if (split_scores) {
        epll_status s = launch_dump_split(g, xhat, H, W, anchors, n, st);
        if (s == EPLL_OK) {
            // band: twice the split form's near-tie threshold (its error bound is half of it)
            int blocks = n < 152 * 2 ? n : 152 * 2;
            if (blocks < 1) blocks = 1;
            EPLL_CU(launch_pdl(k_rescore, dim3(blocks), dim3(32 * RS_WARPS), 0, st, xhat, H, W, anchors, ws.flag, cnt(g, CNT_NFLAG), 0,
                                                        fcap, g->K, g->Rtot, g->d_roff, g->d_r, g->d_B,
                                                        g->d_Blo, g->tab, ws.fscore, 2.0f * tau_abs, 8e-5f,
                                                        ws.kstar, ws.gap, ws.ctr));
            EPLL_LAUNCHED(g);
            return EPLL_OK;
        }
        if (s != EPLL_EUNSUPPORTED) return s;
    }
    for (int f0 = 0; f0 < n; f0 += fcap) {
        const int rows = min(fcap, n - f0);
        const dim3 grid((rows + SEL_THREADS - 1) / SEL_THREADS, g->K < 16 ? g->K : 16);
        EPLL_CU(launch_pdl(k_select_fp32<true>, dim3(grid), dim3(SEL_THREADS), 0, st, 
            xhat, H, W, anchors, 0, g->d_B, g->Rtot, g->d_colk, g->tab, 0.0f, 0.0f, nullptr, nullptr,
            nullptr, nullptr, ws.flag, cnt(g, CNT_NFLAG), f0, fcap, g->K, g->d_roff, ws.fscore));
        EPLL_LAUNCHED(g);
        int blocks = rows < 152 * 2 ? rows : 152 * 2;
        if (blocks < 1) blocks = 1;
        EPLL_CU(launch_pdl(k_rescore, dim3(blocks), dim3(32 * RS_WARPS), 0, st, xhat, H, W, anchors, ws.flag, cnt(g, CNT_NFLAG), f0,
                                                    fcap, g->K, g->Rtot, g->d_roff, g->d_r, g->d_B,
                                                    g->d_Blo, g->tab, ws.fscore, RESCORE_ABS, RESCORE_REL,
                                                    ws.kstar, ws.gap, ws.ctr));
        EPLL_LAUNCHED(g);
    }
    return EPLL_OK;
}

// Component indices handed in by the caller (teacher forcing) are clamped
// into range before they index anything.
// Bucket of a key: negative keys are absent (-1); keys past the range are clamped.
__device__ __forceinline__ int clamp_k(int k, int K) { return k < 0 ? -1 : (k >= K ? K - 1 : k); }

// ============================================================================
// Grouping by component (counting sort): histogram, exclusive scan, scatter,
// in one launch of one thread-block cluster (16 CTAs where the device allows
// it, else 8).  Each CTA counts the keys of its slice in shared memory; after
// a cluster barrier every CTA reads all histograms through distributed shared
// memory, scans the totals over the components and places its own slice
// after the lower-ranked CTAs' entries of each component; CTA 0 also writes
// the work items.  The order inside a group does not matter: every patch's
// estimate depends only on the patch and its component.
// ============================================================================
constexpr int EST_T = 128;  // patches per work item
constexpr int GRP_THREADS = 1024;

// Exclusive block-wide scans of two integers (fixed order); totals in *ta, *tb.
__device__ void block_scan2(int a, int b, int &ea, int &eb, int &ta, int &tb)
{
    __shared__ int wa[GRP_THREADS / 32], wb[GRP_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int ia = a, ib = b;
    for (int o = 1; o < 32; o <<= 1) {
        const int va = __shfl_up_sync(0xffffffffu, ia, o), vb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += va;
            ib += vb;
        }
    }
    if (lane == 31) {
        wa[wid] = ia;
        wb[wid] = ib;
    }
    __syncthreads();
    if (wid == 0) {
        int xa = wa[lane], xb = wb[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int va = __shfl_up_sync(0xffffffffu, xa, o), vb = __shfl_up_sync(0xffffffffu, xb, o);
            if (lane >= o) {
                xa += va;
                xb += vb;
            }
        }
        wa[lane] = xa;
        wb[lane] = xb;
    }
    __syncthreads();
    const int pa = wid ? wa[wid - 1] : 0, pb = wid ? wb[wid - 1] : 0;
    ea = pa + ia - a;
    eb = pb + ib - b;
    ta = wa[31];
    tb = wb[31];
    __syncthreads();
}

__global__ void __launch_bounds__(GRP_THREADS, 1)
k_group(const int *__restrict__ keys, int n, int K, const int *__restrict__ n_dev, int mult,
        int *__restrict__ perm, int4 *__restrict__ items)
{
    pdl_enter();
    namespace cgx = cooperative_groups;
    cgx::cluster_group cl = cgx::this_cluster();
    extern __shared__ int gsh[];
    int *hist = gsh, *base = gsh + K;
    const int rank = (int)cl.block_rank(), nb = (int)cl.num_blocks();
    if (n_dev) n = min(n, mult * *n_dev);
    const int chunk = (n + nb - 1) / nb;
    const int i0 = min(n, rank * chunk), i1 = min(n, i0 + chunk);
    for (int k = threadIdx.x; k < K; k += GRP_THREADS) hist[k] = 0;
    __syncthreads();
    for (int i = i0 + threadIdx.x; i < i1; i += GRP_THREADS) {
        const int k = clamp_k(keys[i], K);
        if (k >= 0) atomicAdd(&hist[k], 1);
    }
    cl.sync();
    int carry = 0, icarry = 0;
    for (int b0 = 0; b0 < K; b0 += GRP_THREADS) {
        const int k = b0 + threadIdx.x;
        int tot = 0, below = 0;
        if (k < K)
            for (int r = 0; r < nb; ++r) {
                const int v = cl.map_shared_rank(hist, r)[k];
                tot += v;
                below += r < rank ? v : 0;
            }
        const int nv = (tot + EST_T - 1) / EST_T;
        int et, ev, tt, tv;
        block_scan2(tot, nv, et, ev, tt, tv);
        if (k < K) {
            const int start = carry + et;
            base[k] = start + below;
            if (rank == 0) {
                const int item0 = icarry + ev;
                for (int t = 0; t < nv; ++t)
                    items[1 + item0 + t] = make_int4(k, start + t * EST_T, min(EST_T, tot - t * EST_T), 0);
            }
        }
        carry += tt;
        icarry += tv;
    }
    if (rank == 0 && threadIdx.x == 0) items[0] = make_int4(0, 0, 0, icarry);
    cl.sync();  // every CTA has read the others' histograms; base[] is local from here on
    for (int i = i0 + threadIdx.x; i < i1; i += GRP_THREADS) {
        const int k = clamp_k(keys[i], K);
        if (k >= 0) perm[atomicAdd(&base[k], 1)] = i;
    }
}

// Cluster size of the grouping kernel (16 where one such cluster fits with
// the largest key range's shared memory, else 8).
static int group_cluster_size()
{
    static int size = 0;
    if (size) return size;
    size = 8;
    const int smem = 2 * 4096 * (int)sizeof(int);
    cudaFuncSetAttribute(k_group, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (cudaFuncSetAttribute(k_group, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(GRP_THREADS);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_group, &cfg) == cudaSuccess && nclusters > 0) size = 16;
    }
    cudaGetLastError();
    return size;
}

void group_setup() { (void)group_cluster_size(); }

// ============================================================================
// Patch estimation (Eqs. 15-16): chat_j = (gamma_j - gamma_P) c_j,
// zhat = Ubar chat + gamma_P z + mean.  A block takes one work item: up to
// 128 patches that selected the same component k.  With the patches Z
// (128 x 64) and Ubar_k in shared memory the two products are register-tiled
// FP32 GEMMs, C = Z Ubar_k and Zhat = C' Ubar_k^T + gamma_P Z: each thread owns
// an 8 x 8 block of outputs and does 64 FMAs per 4 vector loads.  The sums
// run in the order of the definitions (c_j over the pixels in order, zhat_e
// from gamma_P z_e over the coefficients in order).  The estimate is written
// as a 64-float row at each patch's anchor.
// ============================================================================
constexpr int EST_LDZ = EST_T + 4;  // padded patch-major rows

struct EstSmem {
    float Zt[PD][EST_LDZ];  // Zt[e][p]: DC-free patches, transposed
    float Ct[PD][EST_LDZ];  // Ct[j][p]: shrunk coefficients
    float Us[PD][PD];       // Us[e][j], zero beyond the rank
    float Ut[PD][PD];       // Ut[j][e]
    float mus[EST_T];
    float gws[PD];
    int anchor[EST_T];
    int patch[EST_T];  // index in the subset
};

__global__ void __launch_bounds__(EST_T)
k_estimate(const float *__restrict__ xhat, int H, int W, const int *__restrict__ anchors,
           const int *__restrict__ perm, const int4 *__restrict__ items, int Rtot,
           const int *__restrict__ roff, const int *__restrict__ rk_, const float *__restrict__ B,
           Tables tab, float *__restrict__ zrow, int *__restrict__ inv)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char est_raw[];
    EstSmem &sm = *reinterpret_cast<EstSmem *>(est_raw);
    if ((int)blockIdx.x >= items[0].w) return;
    const int4 it = items[1 + blockIdx.x];
    const int k = it.x, first = it.y, cnt_p = it.z;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int o = roff[k], r = rk_[k];
    if (tid < cnt_p) {
        const int i = perm[first + tid];
        sm.anchor[tid] = anchors ? anchors[i] : i;
        sm.patch[tid] = i;
        inv[sm.anchor[tid]] = i;
    }
    for (int idx = tid; idx < PD * PD; idx += EST_T) {
        const int e = idx >> 6, j = idx & 63;
        const float u = j < r ? B[(size_t)e * Rtot + o + j] : 0.0f;
        sm.Us[e][j] = u;
        sm.Ut[j][e] = u;
    }
    if (tid < PD) sm.gws[tid] = tid < r ? tab.gw[o + tid] : 0.0f;
    __syncthreads();
    // gather: each warp takes 32 patches, four at a time (8 loads in flight per lane)
    for (int p0 = w * 32; p0 < w * 32 + 32; p0 += 4) {
        float x0[4], x1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x0[u] = x1[u] = 0.0f;
            if (p0 + u < cnt_p) {
                const int a = sm.anchor[p0 + u];
                const int ai = a / W, aj = a % W;
                x0[u] = xhat[pix(ai, aj, lane >> 3, lane & 7, H, W)];
                x1[u] = xhat[pix(ai, aj, (lane >> 3) + 4, lane & 7, H, W)];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = p0 + u;
            const float m = warp_sum(x0[u] + x1[u]) * (1.0f / PD);
            sm.Zt[lane][p] = p < cnt_p ? x0[u] - m : 0.0f;
            sm.Zt[lane + 32][p] = p < cnt_p ? x1[u] - m : 0.0f;
            if (lane == 0) sm.mus[p] = m;
        }
    }
    __syncthreads();
    const int pg = tid >> 3;  // patches 8 pg .. 8 pg + 7
    const int cg = tid & 7;   // columns (then pixels) 8 cg .. 8 cg + 7
    // ---- C = Z Ubar_k (only column groups below the rank)
    if (8 * cg < r) {
        float acc[8][8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
#pragma unroll 4
        for (int e = 0; e < PD; ++e) {
            const float4 z0 = *reinterpret_cast<const float4 *>(&sm.Zt[e][8 * pg]);
            const float4 z1 = *reinterpret_cast<const float4 *>(&sm.Zt[e][8 * pg + 4]);
            const float4 u0 = *reinterpret_cast<const float4 *>(&sm.Us[e][8 * cg]);
            const float4 u1 = *reinterpret_cast<const float4 *>(&sm.Us[e][8 * cg + 4]);
            const float zv[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
            const float uv[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(zv[a], uv[b], acc[a][b]);
        }
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const float gw = sm.gws[8 * cg + b];
            *reinterpret_cast<float4 *>(&sm.Ct[8 * cg + b][8 * pg]) =
                make_float4(gw * acc[0][b], gw * acc[1][b], gw * acc[2][b], gw * acc[3][b]);
            *reinterpret_cast<float4 *>(&sm.Ct[8 * cg + b][8 * pg + 4]) =
                make_float4(gw * acc[4][b], gw * acc[5][b], gw * acc[6][b], gw * acc[7][b]);
        }
    }
    __syncthreads();
    // ---- Zhat = gamma_P Z + C' Ubar_k^T, plus the mean
    {
        const float gp = tab.gp[k];
        float acc[8][8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const float4 z0 = *reinterpret_cast<const float4 *>(&sm.Zt[8 * cg + b][8 * pg]);
            const float4 z1 = *reinterpret_cast<const float4 *>(&sm.Zt[8 * cg + b][8 * pg + 4]);
            acc[0][b] = gp * z0.x; acc[1][b] = gp * z0.y; acc[2][b] = gp * z0.z; acc[3][b] = gp * z0.w;
            acc[4][b] = gp * z1.x; acc[5][b] = gp * z1.y; acc[6][b] = gp * z1.z; acc[7][b] = gp * z1.w;
        }
#pragma unroll 4
        for (int j = 0; j < r; ++j) {
            const float4 c0 = *reinterpret_cast<const float4 *>(&sm.Ct[j][8 * pg]);
            const float4 c1 = *reinterpret_cast<const float4 *>(&sm.Ct[j][8 * pg + 4]);
            const float4 u0 = *reinterpret_cast<const float4 *>(&sm.Ut[j][8 * cg]);
            const float4 u1 = *reinterpret_cast<const float4 *>(&sm.Ut[j][8 * cg + 4]);
            const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
            const float uv[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(uv[b], cv[a], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int p = 8 * pg + a;
            if (p < cnt_p) {
                const float mu = sm.mus[p];
                float4 *dst = reinterpret_cast<float4 *>(zrow + ((size_t)cg * H * W + sm.patch[p]) * PS);
                dst[0] = make_float4(acc[a][0] + mu, acc[a][1] + mu, acc[a][2] + mu, acc[a][3] + mu);
                dst[1] = make_float4(acc[a][4] + mu, acc[a][5] + mu, acc[a][6] + mu, acc[a][7] + mu);
            }
        }
    }
}

epll_status group_by_component(epll_gmm *g, const int *keys, int n, int *perm, int4 *items, cudaStream_t st,
                               const int *n_dev, int mult)
{
    return group_by_key(g, keys, n, g->K, g->ws.counts, perm, items, st, n_dev, mult);
}

epll_status group_by_key(epll_gmm *g, const int *keys, int n, int K, int *counts, int *perm, int4 *items,
                         cudaStream_t st, const int *n_dev, int mult)
{
    (void)counts;
    if (K > 4096) return fail(EPLL_EUNSUPPORTED, "grouping supports at most 4096 keys");
    const int cl = group_cluster_size();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(GRP_THREADS);
    cfg.dynamicSmemBytes = 2 * (size_t)K * sizeof(int);
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = t_pdl ? 2 : 1;
    EPLL_CU(cudaLaunchKernelEx(&cfg, k_group, keys, n, K, n_dev, mult, perm, items));
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

epll_status launch_estimate(epll_gmm *g, const float *xhat, int H, int W, const int *anchors,
                            int n, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int K = g->K;
    epll_status gs = group_by_component(g, ws.kstar, n, ws.perm, ws.items, st);
    if (gs) return gs;
    static bool attr = false;
    if (!attr) {
        EPLL_CU(cudaFuncSetAttribute(k_estimate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(EstSmem)));
        attr = true;
    }
    const int max_items = (n + EST_T - 1) / EST_T + K;
    EPLL_CU(launch_pdl(k_estimate, dim3(max_items), dim3(EST_T), sizeof(EstSmem), st, xhat, H, W, anchors, ws.perm, ws.items, g->Rtot,
                                                          g->d_roff, g->d_r, g->d_B, g->tab, ws.zrow, ws.inv));
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

// ============================================================================
// Patch reprojection (Algorithm 1; Eq. 6 with the per-pixel patch count),
// written as a gather: every pixel sums, in a fixed order, the estimates of
// the sampled patches that cover it (weighted by their multiplicity in the
// subset), divides by their number, and keeps the current estimate where no
// sampled patch covers it.  Optionally fused with the pixelwise image update
// xhat = (a y + bs xtilde) / (a^2 + bs), bs = beta sigma^2 = lambda * mult
// (with the `valid` boundary bs is weighed by the pixel's patch count / P).
//
// The estimates are stored by patch row: plane u holds, for every sampled
// patch, the 8 estimates of its patch row u at the patch's index in the
// subset (zrow[(u N + i) 8 + v]; the estimation also records i at the
// patch's anchor).  The subsets list their anchors in increasing order (the
// jittered grid nearly so), so the sampled anchors of one anchor row have
// consecutive indices and the estimates that land on one image row from one
// anchor row are contiguous, and the planes are dense (a 1/3 subset fills a
// third of the buffer, which stays in L2).
// A warp owns AG_SPAN = 24 consecutive pixels (i, j0 .. j0 + 23) of R image
// rows; lane l stands for anchor column j0 - 7 + l.  For each anchor row the
// lane loads its multiplicity and, where the anchor is sampled, the 32-byte
// segment of each patch row that lands on one of the warp's image rows
// (coalesced: consecutive lanes, consecutive segments), and adds it to eight
// per-lane sums, one per column offset v.  The multiplicities of all anchor
// rows are loaded before any segment, and the segments of four anchor rows
// at a time, so a warp waits for a few memory round trips, not one per row.  A pixel's value is then the sum
// over v of lane (l - v)'s sum v, gathered with seven shuffles; its count is
// an 8-wide sliding sum of the lanes' multiplicity sums (three shuffles).
// Summation order per pixel: anchor rows ascending, then v ascending.
// ============================================================================
constexpr int AG_SPAN = 32 - (PS - 1);  // output pixels per warp
constexpr int AG_THREADS = 256;

template <int R>
__global__ void __launch_bounds__(AG_THREADS)
k_aggregate(const float *__restrict__ zrow, const unsigned *__restrict__ mult, const int *__restrict__ inv,
            const float *xhat, int H, int W, const float *__restrict__ y,
            const float *__restrict__ a, const float *__restrict__ lamf, float bmult,
            float *xout, int weighted, float *__restrict__ wout)
{
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int gw = (W + AG_SPAN - 1) / AG_SPAN, gh = (H + R - 1) / R;
    const int wid = (int)((blockIdx.x * (unsigned)AG_THREADS + threadIdx.x) >> 5);
    if (wid >= gh * gw) return;  // the whole warp leaves together
    const int i0 = (wid / gw) * R, j0 = (wid % gw) * AG_SPAN;
    int c = (j0 - (PS - 1) + lane) % W;  // >= -7 >= -W
    if (c < 0) c += W;
    const size_t N = (size_t)H * W;
    float V[R][PS];
    unsigned M[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        M[r] = 0u;
#pragma unroll
        for (int v = 0; v < PS; ++v) V[r][v] = 0.0f;
    }
    // anchor rows i0 - 7 .. i0 + R - 1; image row i0 + r takes patch row
    // u = r + 7 - e of anchor row e (0 <= u < 8).  All multiplicities are
    // loaded first, then the sampled segments AG_CHUNK anchor rows at a time
    // (their loads issued together), then added in ascending anchor-row order.
    constexpr int NE = PS + R - 1;
    size_t ab[NE];  // the anchor's patch index in the subset (the anchor itself for the full set)
    unsigned m[NE];
    int ai = (i0 - (PS - 1)) % H;  // >= -7 >= -H
    if (ai < 0) ai += H;
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        const size_t a = (size_t)ai * W + c;
        m[e] = mult ? mult[a] : 1u;
        ab[e] = a;
        if (mult) {
            const int pi = inv[a];
            ab[e] = m[e] ? (size_t)pi : 0;
        }
        if (++ai == H) ai = 0;
    }
    constexpr int AG_CHUNK = 4;
#pragma unroll
    for (int e0 = 0; e0 < NE; e0 += AG_CHUNK) {
        float4 s[AG_CHUNK][R][2];
#pragma unroll
        for (int de = 0; de < AG_CHUNK; ++de) {
            const int e = e0 + de;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int u = r + (PS - 1) - e;
                s[de][r][0] = s[de][r][1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (e < NE && u >= 0 && u < PS && m[e]) {
                    const float4 *src = reinterpret_cast<const float4 *>(zrow + ((size_t)u * N + ab[e]) * PS);
                    s[de][r][0] = src[0];
                    s[de][r][1] = src[1];
                }
            }
        }
#pragma unroll
        for (int de = 0; de < AG_CHUNK; ++de) {
            const int e = e0 + de;
            if (e >= NE) break;
            const float fm = (float)m[e];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int u = r + (PS - 1) - e;
                if (u < 0 || u >= PS) continue;
                M[r] += m[e];
                const float4 s0 = s[de][r][0], s1 = s[de][r][1];
                V[r][0] = fmaf(fm, s0.x, V[r][0]);
                V[r][1] = fmaf(fm, s0.y, V[r][1]);
                V[r][2] = fmaf(fm, s0.z, V[r][2]);
                V[r][3] = fmaf(fm, s0.w, V[r][3]);
                V[r][4] = fmaf(fm, s1.x, V[r][4]);
                V[r][5] = fmaf(fm, s1.y, V[r][5]);
                V[r][6] = fmaf(fm, s1.z, V[r][6]);
                V[r][7] = fmaf(fm, s1.w, V[r][7]);
            }
        }
    }
    const float bs = y ? lamf[0] * bmult : 0.0f;
    const int j = j0 + lane - (PS - 1);  // pixel of this lane (lanes 7 .. 30)
    const bool out_lane = lane >= PS - 1 && lane < PS - 1 + AG_SPAN && j < W;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        // pixel j gets element v of anchor column j - v, held by lane l - v
        float sum = V[r][0];
#pragma unroll
        for (int v = 1; v < PS; ++v) sum += __shfl_up_sync(0xffffffffu, V[r][v], v);
        unsigned cnt = M[r];
        cnt += __shfl_up_sync(0xffffffffu, cnt, 1);
        cnt += __shfl_up_sync(0xffffffffu, cnt, 2);
        cnt += __shfl_up_sync(0xffffffffu, cnt, 4);  // lanes >= 7: anchor columns l - 7 .. l
        const int i = i0 + r;
        if (!out_lane || i >= H) continue;
        const size_t p = (size_t)i * W + j;
        const float xt = cnt ? sum / (float)cnt : xhat[p];
        const float wt = (float)cnt * (1.0f / (float)PD);  // patch count / P
        if (wout) wout[p] = wt;
        if (y) {
            const float ap = a ? a[p] : 1.0f;
            const float bw = weighted ? bs * wt : bs;
            xout[p] = (ap * y[p] + bw * xt) / (ap * ap + bw);
        } else {
            xout[p] = xt;
        }
    }
}

epll_status launch_aggregate(epll_gmm *g, const float *xhat, int H, int W, const unsigned *mult,
                             const float *y, const float *a, const float *lamf, double bmult,
                             float *xout, cudaStream_t st, int weighted, float *wout)
{
    const int R = g->tile_agg == 2 ? 2 : 1;
    const long long warps = (long long)((H + R - 1) / R) * ((W + AG_SPAN - 1) / AG_SPAN);
    const unsigned blocks = (unsigned)((warps * 32 + AG_THREADS - 1) / AG_THREADS);
    if (R == 2)
        EPLL_CU(launch_pdl(k_aggregate<2>, dim3(blocks), dim3(AG_THREADS), 0, st, g->ws.zrow, mult, g->ws.inv, xhat, H, W, y, a, lamf, (float)bmult,
                                                     xout, weighted, wout));
    else
        EPLL_CU(launch_pdl(k_aggregate<1>, dim3(blocks), dim3(AG_THREADS), 0, st, g->ws.zrow, mult, g->ws.inv, xhat, H, W, y, a, lamf, (float)bmult,
                                                     xout, weighted, wout));
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

}  // namespace epll
