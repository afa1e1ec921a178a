// Per-iteration preparation kernels: the FP64 per-beta tables of the
// Gaussian selection / patch estimation steps, and the patch samplers.
#include "epll_internal.cuh"

#include <cuda_fp16.h>
#include <cuda_fp8.h>

namespace epll {

// ============================================================================
// Per-beta tables (Sec. "Complexity via eigenspace implementation", Eq. 8;
// flat-tail form Eqs. 14-16).  One block per component, 64 threads; FP64
// throughout, results rounded to float (plus the float rounding error for the
// compensated rescoring).  1/beta = sigma^2 / (lambda * mult) with lambda read
// from device memory, or 1/beta_direct when beta_direct > 0.
// ============================================================================
__device__ double block64_sum(double v, double *red)
{
    int j = threadIdx.x;
    red[j] = v;
    __syncthreads();
    for (int s = 32; s > 0; s >>= 1) {
        if (j < s) red[j] += red[j + s];
        __syncthreads();
    }
    double tot = red[0];
    __syncthreads();
    return tot;
}

// -2 log w_k + sum_{j<r} log(S_kj + ib) + (P - r) log(lambda_k + ib)
__device__ double component_constant(int k, const int *r, const double *S, const double *w,
                                     const double *lam, double ib, double *red)
{
    int j = threadIdx.x;
    int rk = r[k];
    double v = (j < rk) ? log(S[(size_t)k * PD + j] + ib) : 0.0;
    double c = block64_sum(v, red) - 2.0 * log(w[k]);
    if (rk < PD) c += (double)(PD - rk) * log(lam[k] + ib);
    return c;
}

struct Mults {
    double m[TB_MAX];
};

// Grid (K, nb): component k of batch slot blockIdx.y.
__global__ void __launch_bounds__(64)
k_tables(int K, int Rtot, int Rp, const int *__restrict__ r, const int *__restrict__ roff,
         const double *__restrict__ S, const double *__restrict__ w, const double *__restrict__ lam,
         const double *__restrict__ d_lambda, Mults mults, double sigma2, double beta_direct,
         const float *__restrict__ B, Tables tab0, int fmt)
{
    __shared__ double red[64];
    __shared__ float sq[64 + RTOT_ALIGN];
    __shared__ float tile[PD][PD + 1];  // one 64-column chunk of the basis, padded rows
    const int k = blockIdx.x, j = threadIdx.x;
    const Tables tab = slot_tables(tab0, blockIdx.y, K, Rp, Rtot);
    const double mult = mults.m[blockIdx.y];
    const double ib = beta_direct > 0.0 ? 1.0 / beta_direct : sigma2 / (d_lambda[0] * mult);

    const double c0 = component_constant(0, r, S, w, lam, ib, red);
    const double ck = component_constant(k, r, S, w, lam, ib, red);
    const int rk = r[k];
    const double nuP = lam[k] + ib;
    const double t = rk < PD ? 1.0 / nuP : 0.0;
    const double gP = rk < PD ? lam[k] / nuP : 0.0;
    if (j == 0) {
        double cst = ck - c0;
        float h = (float)cst;
        tab.cst_hi[k] = h;
        tab.cst_lo[k] = (float)(cst - (double)h);
        float th = (float)t;
        tab.t_hi[k] = th;
        tab.t_lo[k] = (float)(t - (double)th);
        tab.gp[k] = (float)gP;
        tab.sgn[k] = rk < PD ? -1.0f : 1.0f;
        if (k == 0) tab.ibeta[0] = (float)ib;
        // error scale of the score: largest 1/nu of this component
        const double numin = rk < PD ? nuP : S[(size_t)k * PD + PD - 1] + ib;
        atomicMax(reinterpret_cast<int *>(tab.tmax), __float_as_int((float)(1.0 / numin)));
    }
    const int o = roff[k], rp = roff[k + 1] - o;
    for (int jj = j; jj < rp; jj += 64) {
        double q = 0.0, gw = 0.0;
        if (jj < rk) {
            double nu = S[(size_t)k * PD + jj] + ib;
            q = 1.0 / nu - t;
            gw = S[(size_t)k * PD + jj] / nu - gP;
        }
        float qh = (float)q;
        tab.q_hi[o + jj] = qh;
        tab.q_lo[o + jj] = (float)(q - (double)qh);
        tab.gw[o + jj] = (float)gw;
        sq[jj] = (float)sqrt(fabs(q));
    }
    if (!fmt) return;
    __syncthreads();
    float s8 = 1.0f;
    if (fmt & 8) {
        // per-component scale of the E4M3 basis: the largest |value| maps to 448
        float m = 0.0f;
        for (int jj = 0; jj < rk; ++jj) m = fmaxf(m, fabsf(B[(size_t)j * Rtot + o + jj] * sq[jj]));
        red[j] = m;
        __syncthreads();
        for (int st = 32; st > 0; st >>= 1) {
            if (j < st) red[j] = fmax(red[j], red[j + st]);
            __syncthreads();
        }
        s8 = red[0] > 0.0 ? (float)red[0] / 448.0f : 1.0f;
        if (j == 0) tab.k8s2[k] = s8 * s8;
    }
    // scaled basis, K-major: B[col][e] = 16-bit(U[e][col] * sqrt|q_col|); the
    // split form stores the BF16 value and the BF16 remainder.  B is e-major,
    // so 64-column chunks go through shared memory: read along the columns
    // (coalesced), written along e (coalesced).
    for (int c0 = 0; c0 < rp; c0 += PD) {
        __syncthreads();  // the previous chunk's reads of tile are done
#pragma unroll 8
        for (int e = 0; e < PD; ++e) {
            const int jj = c0 + j;
            tile[e][j] = (jj < rk) ? B[(size_t)e * Rtot + o + jj] : 0.0f;
        }
        __syncthreads();
        const int nc = min(PD, rp - c0);
        for (int jl = 0; jl < nc; ++jl) {
            const int jj = c0 + jl;
            const float v = (jj < rk) ? tile[j][jl] * sq[jj] : 0.0f;
            const size_t dst = (size_t)(o + jj) * PD + j;
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            if (fmt & 1) tab.B1[dst] = __bfloat16_as_ushort(h);
            if (fmt & 2) tab.B1[dst] = __half_as_ushort(__float2half_rn(v));
            if (fmt & 4) {
                tab.Bs[dst] = __bfloat16_as_ushort(h);
                tab.Bs_lo[dst] = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(h)));
            }
            if (fmt & 8) tab.B8[dst] = (uint8_t)__nv_cvt_float_to_fp8(v / s8, __NV_SATFINITE, __NV_E4M3);
        }
    }
}

epll_status launch_tables(epll_gmm *g, const double *d_lambda, const double *mult, int nb,
                          double sigma2, double beta_direct, int fmt, cudaStream_t st)
{
    Mults m{};
    for (int b = 0; b < nb; ++b) m.m[b] = mult[b];
    EPLL_CU(cudaMemsetAsync(g->tab0.tmax, 0, sizeof(float) * nb, st));
    k_tables<<<dim3(g->K, nb), 64, 0, st>>>(g->K, g->Rtot, g->Rp, g->d_r, g->d_roff, g->d_S, g->d_w,
                                            g->d_lam, d_lambda, m, sigma2, beta_direct, g->d_B, g->tab0, fmt);
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

// ============================================================================
// Counter-based random numbers: splitmix64 (Steele, Lea & Flood, OOPSLA 2014;
// output-function constants of Vigna's public-domain splitmix64.c).
// Draw idx of stream s for seed x: state = mix(x + (s+1) G), draw = mix(state + (idx+1) G).
// ============================================================================
__device__ __forceinline__ uint64_t smix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
constexpr uint64_t GOLDEN = 0x9e3779b97f4a7c15ULL;

__device__ __forceinline__ uint64_t stream_state(uint64_t seed, uint64_t s)
{
    return smix(seed + (s + 1) * GOLDEN);
}
__device__ __forceinline__ uint64_t draw(uint64_t state, uint64_t idx)
{
    return smix(state + (idx + 1) * GOLDEN);
}
__device__ __forceinline__ int uniform_int(uint64_t u, int m)
{
    return (int)(((u >> 32) * (uint64_t)m) >> 32);
}

// ---------------------------------------------------------------- jitter
// Jittered grid of Eq. 20: spacing s, global shift from draws 0/1, per-point
// offsets in [-J, J] from draws 2+2g / 3+2g; raster order of grid points.
// regular != 0: the regular grid of the same spacing (Sec. "Speed-up via the
// restriction to a random subset of patches"): no shift, no offsets.
__global__ void k_jitter(int H, int W, int s, uint64_t seed, int t0, int ni, int nj, int regular,
                         int *__restrict__ anchors_all, unsigned *__restrict__ mult_all)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ni * nj) return;
    const int t = t0 + blockIdx.y;
    int *anchors = anchors_all + (size_t)blockIdx.y * H * W;
    unsigned *mult = mult_all + (size_t)blockIdx.y * H * W;
    const uint64_t st = stream_state(seed, (uint64_t)t);
    const int J = regular ? 0 : (PS - s) / 2;
    const int gi = regular ? 0 : uniform_int(draw(st, 0), s), gj = regular ? 0 : uniform_int(draw(st, 1), s);
    const int n = g / nj, m = g % nj;
    const int di = regular ? 0 : uniform_int(draw(st, 2 + 2 * (uint64_t)g), 2 * J + 1) - J;
    const int dj = regular ? 0 : uniform_int(draw(st, 3 + 2 * (uint64_t)g), 2 * J + 1) - J;
    const int i = ((gi + s * n + di) % H + H) % H;
    const int j = ((gj + s * m + dj) % W + W) % W;
    const int a = i * W + j;
    anchors[g] = a;
    atomicAdd(&mult[a], 1u);
}

// ---------------------------------------------------------------- fraction
// Exactly M = ceil(frac N) anchors: those with the smallest (key, anchor),
// key = high 32 bits of draw(anchor).  A 4-pass radix select (8-bit digits,
// most significant first) finds the key of rank M-1 and its rank among equal
// keys; a 3-phase stream compaction then writes the selection in anchor order.
// sel = {prefix, mask, rank} of the partially determined threshold key.
__device__ __forceinline__ uint32_t frac_key(uint64_t st, int a)
{
    return (uint32_t)(draw(st, (uint64_t)a) >> 32);
}

// Scratch of batch slot b (t = t0 + b) starts at scratch + b * sstride:
// [0, 1024) histograms of the 4 passes, [1024, 1027) sel, from 1040 the tiles.
__global__ void __launch_bounds__(256)
k_frac_hist(int N, uint64_t seed, int t0, int pass, unsigned *__restrict__ scratch, size_t sstride)
{
    __shared__ unsigned h[256];
    const int t = t0 + blockIdx.y;
    unsigned *hist = scratch + blockIdx.y * sstride;
    const unsigned *sel = hist + 1024;
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t st = stream_state(seed, (uint64_t)t);
    const int shift = 24 - 8 * pass;
    const unsigned prefix = pass ? sel[0] : 0u, mask = pass ? sel[1] : 0u;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
        uint32_t key = frac_key(st, a);
        if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[pass * 256 + threadIdx.x], h[threadIdx.x]);
}

__global__ void __launch_bounds__(256)
k_frac_pick(int pass, int M, unsigned *__restrict__ scratch, size_t sstride)
{
    __shared__ unsigned c[256];
    const unsigned *hist = scratch + blockIdx.y * sstride;
    unsigned *sel = scratch + blockIdx.y * sstride + 1024;
    const int d = threadIdx.x;
    const unsigned hd = hist[pass * 256 + d];
    c[d] = hd;
    __syncthreads();
    // inclusive scan (Hillis-Steele)
    for (int off = 1; off < 256; off <<= 1) {
        unsigned v = d >= off ? c[d - off] : 0u;
        __syncthreads();
        c[d] += v;
        __syncthreads();
    }
    const unsigned before = c[d] - hd;
    const unsigned R = pass ? sel[2] : (unsigned)(M - 1);
    const unsigned prefix = pass ? sel[0] : 0u, mask = pass ? sel[1] : 0u;
    __syncthreads();
    if (hd && before <= R && R < before + hd) {
        const int shift = 24 - 8 * pass;
        sel[0] = prefix | ((unsigned)d << shift);
        sel[1] = mask | (255u << shift);
        sel[2] = R - before;
    }
}

// phase 1: per-tile counts of keys below / equal to the threshold
__global__ void __launch_bounds__(256)
k_frac_count(int N, uint64_t seed, int t0, unsigned *__restrict__ scratch, size_t sstride)
{
    __shared__ unsigned long long red[256];
    const int t = t0 + blockIdx.y;
    const unsigned *sel = scratch + blockIdx.y * sstride + 1024;
    unsigned long long *tile = reinterpret_cast<unsigned long long *>(scratch + blockIdx.y * sstride + 1040);
    const uint64_t st = stream_state(seed, (uint64_t)t);
    const uint32_t thr = sel[0];
    unsigned less = 0, eq = 0;
    const int base = blockIdx.x * FRAC_TILE + threadIdx.x * FRAC_ITEMS;
    for (int q = 0; q < FRAC_ITEMS; ++q) {
        int a = base + q;
        if (a < N) {
            uint32_t key = frac_key(st, a);
            less += key < thr;
            eq += key == thr;
        }
    }
    red[threadIdx.x] = ((unsigned long long)less << 32) | eq;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) tile[blockIdx.x] = red[0];
}

// phase 2: exclusive scan of the tile counts (one block)
__global__ void __launch_bounds__(1024)
k_frac_scan(int ntiles, unsigned *__restrict__ scratch, size_t sstride)
{
    unsigned long long *tile = reinterpret_cast<unsigned long long *>(scratch + blockIdx.y * sstride + 1040);
    __shared__ unsigned long long c[1024];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < ntiles; b0 += 1024) {
        int b = b0 + threadIdx.x;
        unsigned long long v = b < ntiles ? tile[b] : 0ull;
        c[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            unsigned long long u = threadIdx.x >= off ? c[threadIdx.x - off] : 0ull;
            __syncthreads();
            c[threadIdx.x] += u;
            __syncthreads();
        }
        if (b < ntiles) tile[b] = carry + c[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += c[1023];
        __syncthreads();
    }
}

// phase 3: write the selected anchors in increasing order
__global__ void __launch_bounds__(256)
k_frac_write(int N, uint64_t seed, int t0, const unsigned *__restrict__ scratch, size_t sstride,
             int *__restrict__ anchors_all, unsigned *__restrict__ mult_all)
{
    __shared__ unsigned long long c[256];
    const int t = t0 + blockIdx.y;
    const unsigned *sel = scratch + blockIdx.y * sstride + 1024;
    const unsigned long long *tile =
        reinterpret_cast<const unsigned long long *>(scratch + blockIdx.y * sstride + 1040);
    int *anchors = anchors_all + (size_t)blockIdx.y * N;
    unsigned *mult = mult_all + (size_t)blockIdx.y * N;
    const uint64_t st = stream_state(seed, (uint64_t)t);
    const uint32_t thr = sel[0];
    const unsigned need = sel[2] + 1u;  // keys equal to thr that are selected
    const int base = blockIdx.x * FRAC_TILE + threadIdx.x * FRAC_ITEMS;
    uint32_t keys[FRAC_ITEMS];
    unsigned less = 0, eq = 0;
    for (int q = 0; q < FRAC_ITEMS; ++q) {
        int a = base + q;
        keys[q] = a < N ? frac_key(st, a) : 0xffffffffu;
        if (a < N) {
            less += keys[q] < thr;
            eq += keys[q] == thr;
        }
    }
    const unsigned long long mine = ((unsigned long long)less << 32) | eq;
    c[threadIdx.x] = mine;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        unsigned long long u = threadIdx.x >= off ? c[threadIdx.x - off] : 0ull;
        __syncthreads();
        c[threadIdx.x] += u;
        __syncthreads();
    }
    unsigned long long before = tile[blockIdx.x] + c[threadIdx.x] - mine;
    unsigned lb = (unsigned)(before >> 32), eb = (unsigned)(before & 0xffffffffu);
    for (int q = 0; q < FRAC_ITEMS; ++q) {
        int a = base + q;
        if (a >= N) break;
        bool take = false;
        if (keys[q] < thr) {
            take = true;
        } else if (keys[q] == thr) {
            take = eb < need;
        }
        if (take) anchors[lb + (eb < need ? eb : need)] = a;
        mult[a] = take ? 1u : 0u;
        lb += keys[q] < thr;
        eb += keys[q] == thr;
    }
}

int sample_count(int H, int W, const epll_options &o)
{
    const int N = H * W;
    if (o.subset == EPLL_SUBSET_FRACTION) {
        int M = (int)ceil(o.subset_param * (double)N);
        return M > N ? N : (M < 1 ? 1 : M);
    }
    if (o.subset == EPLL_SUBSET_JITTER || o.subset == EPLL_SUBSET_REGULAR) {
        int s = (int)o.subset_param;
        return ((H + s - 1) / s) * ((W + s - 1) / s);
    }
    return N;
}

size_t sampler_stride(size_t N) { return sampler_words(N); }

epll_status launch_sample(epll_gmm *g, int H, int W, const epll_options &o, int t0, int nb, int *n,
                          int *anchors, unsigned *mult, unsigned *scratch, size_t sstride,
                          cudaStream_t st)
{
    const int N = H * W;
    *n = sample_count(H, W, o);
    if (o.subset == EPLL_SUBSET_ALL) return EPLL_OK;
    if (o.subset == EPLL_SUBSET_JITTER || o.subset == EPLL_SUBSET_REGULAR) {
        const int s = (int)o.subset_param;
        EPLL_CU(cudaMemsetAsync(mult, 0, sizeof(unsigned) * (size_t)N * nb, st));
        const int ni = (H + s - 1) / s, nj = (W + s - 1) / s;
        k_jitter<<<dim3((ni * nj + 255) / 256, nb), 256, 0, st>>>(
            H, W, s, o.seed, t0, ni, nj, o.subset == EPLL_SUBSET_REGULAR ? 1 : 0, anchors, mult);
        EPLL_LAUNCHED(g);
        return EPLL_OK;
    }
    // FRACTION
    for (int b = 0; b < nb; ++b)
        EPLL_CU(cudaMemsetAsync(scratch + b * sstride, 0, sizeof(unsigned) * 1024, st));
    int hb = (N + 255) / 256;
    if (hb > 152 * 4) hb = 152 * 4;
    for (int pass = 0; pass < 4; ++pass) {
        k_frac_hist<<<dim3(hb, nb), 256, 0, st>>>(N, o.seed, t0, pass, scratch, sstride);
        EPLL_LAUNCHED(g);
        k_frac_pick<<<dim3(1, nb), 256, 0, st>>>(pass, *n, scratch, sstride);
        EPLL_LAUNCHED(g);
    }
    const int ntiles = (N + FRAC_TILE - 1) / FRAC_TILE;
    k_frac_count<<<dim3(ntiles, nb), 256, 0, st>>>(N, o.seed, t0, scratch, sstride);
    EPLL_LAUNCHED(g);
    k_frac_scan<<<dim3(1, nb), 1024, 0, st>>>(ntiles, scratch, sstride);
    EPLL_LAUNCHED(g);
    k_frac_write<<<dim3(ntiles, nb), 256, 0, st>>>(N, o.seed, t0, scratch, sstride, anchors, mult);
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

}  // namespace epll
