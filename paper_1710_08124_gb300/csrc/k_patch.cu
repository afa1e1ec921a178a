// Patch-step kernels of Algorithm 1: patch extraction, Gaussian selection
// (FP32 SIMT form), near-tie rescoring in compensated FP32, grouping of the
// patches by selected component, Wiener patch estimation (Eqs. 15-16) and
// patch reprojection by overlap-add averaging fused with the image update.
#include "epll_internal.cuh"

#include <cfloat>

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
    k_select_fp32<false><<<(n + SEL_THREADS - 1) / SEL_THREADS, SEL_THREADS, 0, st>>>(
        xhat, H, W, anchors, n, g->d_B, g->Rtot, g->d_colk, g->tab, tau_abs, tau_rel, ws.kstar, ws.gap,
        ws.flag, nflag, nullptr, nullptr, 0, 0, g->K, g->d_roff, nullptr);
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
constexpr int RS_WARPS = 4;

// Entries [f0, f0 + fcap) of the near-tie list; scores[(f - f0) * K + k] holds
// each component's FP32 score (written by the FP32 kernel in list mode).
__global__ void __launch_bounds__(32 * RS_WARPS)
k_rescore(const float *__restrict__ xhat, int H, int W, const int *__restrict__ anchors,
          const int *__restrict__ flag, const int *__restrict__ nflag, int f0, int fcap, int K,
          int Rtot, const int *__restrict__ roff, const int *__restrict__ rk_,
          const float *__restrict__ B, const float *__restrict__ Blo, Tables tab,
          const float *__restrict__ scores, float band_abs, float band_rel, int *__restrict__ kstar,
          float *__restrict__ gap, long long *__restrict__ ctr)
{
    __shared__ float zh[RS_WARPS][PD], zl[RS_WARPS][PD];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = min(*nflag - f0, fcap);
    const int gw = blockIdx.x * RS_WARPS + w, nw = gridDim.x * RS_WARPS;
    if (gw == 0 && lane == 0 && total > 0) atomicAdd((unsigned long long *)ctr, (unsigned long long)total);
    for (int f = gw; f < total; f += nw) {
        const int i = flag[f0 + f];
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
        zh[w][lane] = z0.hi; zl[w][lane] = z0.lo;
        zh[w][lane + 32] = z1.hi; zl[w][lane + 32] = z1.lo;
        __syncwarp();
        const float *sc = scores + (size_t)f * K;
        float best = FLT_MAX;
        for (int k = lane; k < K; k += 32) best = fminf(best, sc[k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
        const float band = band_abs + band_rel * (zz.hi + zz.lo) * tab.tmax[0];
        // compensated scores of the components within the band of the best;
        // lanes scan 32 components at a time, a ballot lists the candidates
        df b1 = {FLT_MAX, 0.0f}, b2 = {FLT_MAX, 0.0f};
        int kb = -1;
        float outside = FLT_MAX;
        for (int k0 = 0; k0 < K; k0 += 32) {
            const float sk = k0 + lane < K ? sc[k0 + lane] : FLT_MAX;
            const bool cand = k0 + lane < K && !(sk > best + band);
            if (!cand) outside = fminf(outside, sk);
            unsigned m = __ballot_sync(0xffffffffu, cand);
            while (m) {
                const int k = k0 + __ffs(m) - 1;
                m &= m - 1;
                const int o = roff[k], r = rk_[k];
                df part = {0.0f, 0.0f};
                for (int j = lane; j < r; j += 32) {
                    df c = {0.0f, 0.0f};
                    for (int e = 0; e < PD; ++e) {
                        df u = {B[(size_t)e * Rtot + o + j], Blo[(size_t)e * Rtot + o + j]};
                        c = df_add(c, df_mul(u, {zh[w][e], zl[w][e]}));
                    }
                    df q = {tab.q_hi[o + j], tab.q_lo[o + j]};
                    part = df_add(part, df_mul(q, df_mul(c, c)));
                }
                df sv = df_warp_sum(part);
                sv = df_add(sv, df_mul({tab.t_hi[k], tab.t_lo[k]}, zz));
                sv = df_add(sv, {tab.cst_hi[k], tab.cst_lo[k]});
                if (df_less(sv, b1)) { b2 = b1; b1 = sv; kb = k; }
                else if (df_less(sv, b2)) { b2 = sv; }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) outside = fminf(outside, __shfl_xor_sync(0xffffffffu, outside, o));
        if (lane == 0 && kb >= 0) {  // kb < 0 only if every score was NaN
            kstar[i] = kb;
            float g2 = (b2.hi == FLT_MAX) ? outside - (b1.hi + b1.lo)
                                          : (b2.hi - b1.hi) + (b2.lo - b1.lo);
            gap[i] = fminf(g2, outside - (b1.hi + b1.lo));
        }
        __syncwarp();
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
            int blocks = (n + RS_WARPS - 1) / RS_WARPS;
            if (blocks > 152 * 4) blocks = 152 * 4;
            k_rescore<<<blocks, 32 * RS_WARPS, 0, st>>>(xhat, H, W, anchors, ws.flag, cnt(g, CNT_NFLAG), 0,
                                                        fcap, g->K, g->Rtot, g->d_roff, g->d_r, g->d_B,
                                                        g->d_Blo, g->tab, ws.fscore, 2.0f * tau_abs, 8e-5f,
                                                        ws.kstar, ws.gap, ws.ctr);
            EPLL_LAUNCHED(g);
            return EPLL_OK;
        }
        if (s != EPLL_EUNSUPPORTED) return s;
    }
    for (int f0 = 0; f0 < n; f0 += fcap) {
        const int rows = min(fcap, n - f0);
        const dim3 grid((rows + SEL_THREADS - 1) / SEL_THREADS, g->K < 16 ? g->K : 16);
        k_select_fp32<true><<<grid, SEL_THREADS, 0, st>>>(
            xhat, H, W, anchors, 0, g->d_B, g->Rtot, g->d_colk, g->tab, 0.0f, 0.0f, nullptr, nullptr,
            nullptr, nullptr, ws.flag, cnt(g, CNT_NFLAG), f0, fcap, g->K, g->d_roff, ws.fscore);
        EPLL_LAUNCHED(g);
        int blocks = (rows + RS_WARPS - 1) / RS_WARPS;
        if (blocks > 152 * 4) blocks = 152 * 4;
        k_rescore<<<blocks, 32 * RS_WARPS, 0, st>>>(xhat, H, W, anchors, ws.flag, cnt(g, CNT_NFLAG), f0,
                                                    fcap, g->K, g->Rtot, g->d_roff, g->d_r, g->d_B,
                                                    g->d_Blo, g->tab, ws.fscore, RESCORE_ABS, RESCORE_REL,
                                                    ws.kstar, ws.gap, ws.ctr);
        EPLL_LAUNCHED(g);
    }
    return EPLL_OK;
}

// Component indices handed in by the caller (teacher forcing) are clamped
// into range before they index anything.
__device__ __forceinline__ int clamp_k(int k, int K) { return k < 0 ? 0 : (k >= K ? K - 1 : k); }

// ============================================================================
// Grouping by component (counting sort): histogram, exclusive scan, scatter.
// The order inside a group does not matter: every patch's estimate depends
// only on the patch and its component.
// ============================================================================
__global__ void k_bucket_hist(const int *__restrict__ kstar, int n, int K, int *__restrict__ counts)
{
    extern __shared__ int h[];
    for (int k = threadIdx.x; k < K; k += blockDim.x) h[k] = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(&h[clamp_k(kstar[i], K)], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        if (h[k]) atomicAdd(&counts[k], h[k]);
}

__global__ void __launch_bounds__(1024) k_bucket_scan(int K, int *__restrict__ counts)
{
    // counts[0..K) -> cursors (exclusive prefix), in place
    __shared__ int c[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < K; b0 += 1024) {
        int k = b0 + threadIdx.x;
        int v = k < K ? counts[k] : 0;
        c[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            int u = threadIdx.x >= off ? c[threadIdx.x - off] : 0;
            __syncthreads();
            c[threadIdx.x] += u;
            __syncthreads();
        }
        if (k < K) counts[k] = carry + c[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += c[1023];
        __syncthreads();
    }
}

__global__ void k_bucket_scatter(const int *__restrict__ kstar, int n, int K, int *__restrict__ cursor,
                                 int *__restrict__ perm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = i < n ? clamp_k(kstar[i], K) : -1;
    // lanes with the same component share one atomic: the lowest such lane
    // reserves the group's slots, the others take consecutive ones
    const unsigned peers = __match_any_sync(0xffffffffu, k);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader && k >= 0) base = atomicAdd(&cursor[k], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (k >= 0) perm[base + rank] = i;
}

// ============================================================================
// Patch estimation (Eqs. 15-16): chat_j = (gamma_j - gamma_P) c_j,
// zhat = Ubar chat + gamma_P z + mean.  A block takes 128 consecutive entries
// of the component-grouped list, one patch per thread (the DC-free patch in
// registers).  For every run of equal components in the block's range
// Ubar_k and its transpose are staged in shared memory and read back as
// float4 broadcasts, four FMAs per load, in the order of the definitions
// (c_j sums over the pixels in order, zhat_e starts from gamma_P z_e and adds
// the coefficients in order).  Loops over basis columns stay rolled so the
// kernel fits the instruction cache; the coefficients live in a padded
// per-thread row of shared memory.  The estimate is written as a 64-float
// row at the patch's anchor.
// ============================================================================
constexpr int EST_T = 128;
constexpr int EST_LD = PD + 1;  // padded row: thread t's row hits distinct banks

struct EstSmem {
    union {
        float zs[EST_T][EST_LD];  // gathered DC-free patches (first phase only)
        struct {
            float Us[PD][PD];  // Us[e][j], zero beyond the rank
            float UT[PD][PD];  // UT[j][e]
        } u;
    } a;
    float cs[EST_T][EST_LD];  // shrunk coefficients of each thread's patch
    float mus[EST_T];
    float gws[PD];
    int anchor[EST_T];
    int run_end;
};

__global__ void __launch_bounds__(EST_T, 3)
k_estimate(const float *__restrict__ xhat, int H, int W, const int *__restrict__ anchors, int n,
           const int *__restrict__ perm, const int *__restrict__ kstar, int K, int Rtot,
           const int *__restrict__ roff, const int *__restrict__ rk_, const float *__restrict__ B,
           Tables tab, float *__restrict__ zrow)
{
    extern __shared__ __align__(16) unsigned char est_raw[];
    EstSmem &sm = *reinterpret_cast<EstSmem *>(est_raw);
    const int begin = blockIdx.x * EST_T;
    const int end = min(n, begin + EST_T);
    const int q = begin + threadIdx.x;
    const bool valid = q < end;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (valid) {
        const int i = perm[q];
        sm.anchor[threadIdx.x] = anchors ? anchors[i] : i;
    }
    __syncthreads();
    // each warp gathers its 32 patches four at a time (8 loads in flight per lane)
    const int cnt_p = end - begin;
    for (int p0 = w * 32; p0 < min(cnt_p, w * 32 + 32); p0 += 4) {
        float x0[4], x1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = min(p0 + u, cnt_p - 1);
            const int a = sm.anchor[p];
            const int ai = a / W, aj = a % W;
            x0[u] = xhat[pix(ai, aj, lane >> 3, lane & 7, H, W)];
            x1[u] = xhat[pix(ai, aj, (lane >> 3) + 4, lane & 7, H, W)];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = p0 + u;
            const float m = warp_sum(x0[u] + x1[u]) * (1.0f / PD);
            if (p < cnt_p) {
                sm.a.zs[p][lane] = x0[u] - m;
                sm.a.zs[p][lane + 32] = x1[u] - m;
                if (lane == 0) sm.mus[p] = m;
            }
        }
    }
    __syncthreads();
    int mk = -1, a = 0;
    float z[PD];
    float mu = 0.0f;
    if (valid) {
        mk = clamp_k(kstar[perm[q]], K);
        a = sm.anchor[threadIdx.x];
        mu = sm.mus[threadIdx.x];
#pragma unroll
        for (int e = 0; e < PD; ++e) z[e] = sm.a.zs[threadIdx.x][e];
    }
    __syncthreads();
    int pos = begin;
    while (pos < end) {
        const int k = clamp_k(kstar[perm[pos]], K);
        if (threadIdx.x == 0) sm.run_end = end;
        __syncthreads();
        for (int q2 = pos + threadIdx.x; q2 < end; q2 += EST_T)
            if (clamp_k(kstar[perm[q2]], K) != k) atomicMin(&sm.run_end, q2);
        const int o = roff[k], r = rk_[k];
        for (int idx = threadIdx.x; idx < PD * PD; idx += EST_T) {
            const int e = idx >> 6, j = idx & 63;
            const float u = j < r ? B[(size_t)e * Rtot + o + j] : 0.0f;
            sm.a.u.Us[e][j] = u;
            sm.a.u.UT[j][e] = u;
        }
        if (threadIdx.x < PD) sm.gws[threadIdx.x] = (int)threadIdx.x < r ? tab.gw[o + threadIdx.x] : 0.0f;
        __syncthreads();
        const int stop = sm.run_end;
        if (valid && mk == k) {
            const float gp = tab.gp[k];
            // c_j = Ubar_j . z, four columns per pass
#pragma unroll 1
            for (int j4 = 0; 4 * j4 < r; ++j4) {
                float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
                for (int e = 0; e < PD; ++e) {
                    const float4 u = reinterpret_cast<const float4 *>(&sm.a.u.Us[e][0])[j4];
                    a0 = fmaf(u.x, z[e], a0);
                    a1 = fmaf(u.y, z[e], a1);
                    a2 = fmaf(u.z, z[e], a2);
                    a3 = fmaf(u.w, z[e], a3);
                }
                sm.cs[threadIdx.x][4 * j4 + 0] = sm.gws[4 * j4 + 0] * a0;
                sm.cs[threadIdx.x][4 * j4 + 1] = sm.gws[4 * j4 + 1] * a1;
                sm.cs[threadIdx.x][4 * j4 + 2] = sm.gws[4 * j4 + 2] * a2;
                sm.cs[threadIdx.x][4 * j4 + 3] = sm.gws[4 * j4 + 3] * a3;
            }
            // zhat_e = gamma_P z_e + sum_j Ubar_ej chat_j
            float acc[PD];
#pragma unroll
            for (int e = 0; e < PD; ++e) acc[e] = gp * z[e];
#pragma unroll 1
            for (int j = 0; j < r; ++j) {
                const float cj = sm.cs[threadIdx.x][j];
#pragma unroll
                for (int e4 = 0; e4 < PD / 4; ++e4) {
                    const float4 u = reinterpret_cast<const float4 *>(&sm.a.u.UT[j][0])[e4];
                    acc[4 * e4 + 0] = fmaf(u.x, cj, acc[4 * e4 + 0]);
                    acc[4 * e4 + 1] = fmaf(u.y, cj, acc[4 * e4 + 1]);
                    acc[4 * e4 + 2] = fmaf(u.z, cj, acc[4 * e4 + 2]);
                    acc[4 * e4 + 3] = fmaf(u.w, cj, acc[4 * e4 + 3]);
                }
            }
            float4 *dst = reinterpret_cast<float4 *>(zrow + (size_t)a * PD);
#pragma unroll
            for (int e4 = 0; e4 < PD / 4; ++e4)
                dst[e4] = make_float4(acc[4 * e4] + mu, acc[4 * e4 + 1] + mu, acc[4 * e4 + 2] + mu,
                                      acc[4 * e4 + 3] + mu);
        }
        __syncthreads();
        pos = stop;
    }
}

epll_status launch_estimate(epll_gmm *g, const float *xhat, int H, int W, const int *anchors,
                            int n, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int K = g->K;
    int *counts = ws.counts;  // [K] counts -> cursors
    EPLL_CU(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)K, st));
    int hb = (n + 255) / 256;
    if (hb > 152 * 2) hb = 152 * 2;
    k_bucket_hist<<<hb, 256, sizeof(int) * (size_t)K, st>>>(ws.kstar, n, K, counts);
    EPLL_LAUNCHED(g);
    k_bucket_scan<<<1, 1024, 0, st>>>(K, counts);
    EPLL_LAUNCHED(g);
    k_bucket_scatter<<<(n + 255) / 256, 256, 0, st>>>(ws.kstar, n, K, counts, ws.perm);
    EPLL_LAUNCHED(g);
    static bool attr = false;
    if (!attr) {
        EPLL_CU(cudaFuncSetAttribute(k_estimate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(EstSmem)));
        attr = true;
    }
    k_estimate<<<(n + EST_T - 1) / EST_T, EST_T, sizeof(EstSmem), st>>>(
        xhat, H, W, anchors, n, ws.perm, ws.kstar, K, g->Rtot, g->d_roff, g->d_r, g->d_B, g->tab,
        ws.zrow);
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

// ============================================================================
// Patch reprojection (Algorithm 1; Eq. 6 with the per-pixel patch count),
// written as a gather: every pixel sums, in a fixed order, the estimates of
// the sampled patches that cover it (weighted by their multiplicity in the
// subset), divides by their number, and keeps the current estimate where no
// sampled patch covers it.  Optionally fused with the pixelwise image update
// xhat = (a y + bs xtilde) / (a^2 + bs), bs = beta sigma^2 = lambda * mult.
// ============================================================================
__global__ void __launch_bounds__(256)
k_aggregate(const float *__restrict__ zrow, const unsigned *__restrict__ mult,
            const float *xhat, int H, int W, const float *__restrict__ y,
            const float *__restrict__ a, const double *__restrict__ d_lambda, double bmult,
            float *xout)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= H * W) return;
    const int i = p / W, j = p % W;
    float sum = 0.0f;
    unsigned cnt = 0;
#pragma unroll
    for (int u = 0; u < PS; ++u) {
        int ai = i - u;
        if (ai < 0) ai += H;
#pragma unroll
        for (int v = 0; v < PS; ++v) {
            int aj = j - v;
            if (aj < 0) aj += W;
            const size_t an = (size_t)ai * W + aj;
            const unsigned m = mult ? mult[an] : 1u;
            if (m) {
                sum = fmaf((float)m, zrow[an * PD + u * PS + v], sum);
                cnt += m;
            }
        }
    }
    const float xt = cnt ? sum / (float)cnt : xhat[p];
    if (y) {
        const float bs = (float)(d_lambda[0] * bmult);
        const float ap = a ? a[p] : 1.0f;
        xout[p] = (ap * y[p] + bs * xt) / (ap * ap + bs);
    } else {
        xout[p] = xt;
    }
}

epll_status launch_aggregate(epll_gmm *g, const float *xhat, int H, int W, const unsigned *mult,
                             const float *y, const float *a, const double *d_lambda, double bmult,
                             float *xout, cudaStream_t st)
{
    const int N = H * W;
    k_aggregate<<<(N + 255) / 256, 256, 0, st>>>(g->ws.zrow, mult, xhat, H, W, y, a, d_lambda, bmult,
                                                 xout);
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

}  // namespace epll
