// Per-iteration preparation kernels: the FP64 per-beta tables of the
// Gaussian selection / patch estimation steps, and the patch samplers.
#include "epll_internal.cuh"

#include <cooperative_groups.h>
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
struct Mults {
    double m[TB_MAX];
};

// Grid (K, nb): component k of batch slot blockIdx.y, 64 threads: the
// per-component constants, the per-column q, Wiener gains and basis scale
// sqrt|q|, and (E4M3 basis) the component's scale.
__global__ void __launch_bounds__(64)
k_tables(int K, int Rtot, int Rp, const int *__restrict__ r, const int *__restrict__ roff,
         const double *__restrict__ S, const double *__restrict__ w, const double *__restrict__ lam,
         const double *__restrict__ d_lambda, Mults mults, double sigma2, double beta_direct,
         const float *__restrict__ B, Tables tab0, int fmt)
{
    pdl_enter();
    __shared__ double red[64];
    __shared__ float sq[64 + RTOT_ALIGN];
    __shared__ double s_ib;
    const int k = blockIdx.x, j = threadIdx.x, lane = j & 31;
    const Tables tab = slot_tables(tab0, blockIdx.y, K, Rp, Rtot);
    const int rk = r[k];
    // FP64 arithmetic is scarce on this GPU: block-wide scalars are formed
    // once, and the log-determinant sums from eight partial products each
    if (j < 32) {
        double ib = 0.0;
        if (lane == 0) {
            const double mult = mults.m[blockIdx.y];
            ib = beta_direct > 0.0 ? 1.0 / beta_direct : sigma2 / (d_lambda[0] * mult);
        }
        ib = __shfl_sync(0xffffffffu, ib, 0);
        // lanes 0..7: sum_{j<r_0} log(S_0j + ib) in eight partial products (component 0,
        // whose constant is subtracted from every component's); lanes 8..15: component k;
        // lanes 16..19: log w_0, log w_k, log(lambda_0 + ib), log(lambda_k + ib).
        // A partial product of eight factors rounds by at most 7 ulp, far below the
        // float rounding the tables end in; one outside (1e-300, 1e300) falls back
        // to one logarithm per factor.
        double v = 0.0;
        if (lane < 16) {
            const int c = lane < 8 ? 0 : k, e0 = 8 * (lane & 7), e1 = min(e0 + 8, r[c]);
            double prod = 1.0;
            for (int e = e0; e < e1; ++e) prod *= S[(size_t)c * PD + e] + ib;
            if (prod > 1e-300 && prod < 1e300) {
                v = log(prod);
            } else {
                for (int e = e0; e < e1; ++e) v += log(S[(size_t)c * PD + e] + ib);
            }
        } else if (lane < 20) {
            const int c = (lane & 1) ? k : 0;
            v = log(lane < 18 ? w[c] : lam[c] + ib);
        }
        double sum8 = v;
        sum8 += __shfl_xor_sync(0xffffffffu, sum8, 1);
        sum8 += __shfl_xor_sync(0xffffffffu, sum8, 2);
        sum8 += __shfl_xor_sync(0xffffffffu, sum8, 4);
        const double l0 = __shfl_sync(0xffffffffu, sum8, 0), lk = __shfl_sync(0xffffffffu, sum8, 8);
        const double lw0 = __shfl_sync(0xffffffffu, v, 16), lwk = __shfl_sync(0xffffffffu, v, 17);
        const double ll0 = __shfl_sync(0xffffffffu, v, 18), llk = __shfl_sync(0xffffffffu, v, 19);
        if (lane == 0) {
            // -2 log w + sum_{j<r} log(S_j + ib) + (P - r) log(lambda + ib), component k minus component 0
            const int r0 = r[0];
            double c0 = l0 - 2.0 * lw0, ck = lk - 2.0 * lwk;
            if (r0 < PD) c0 += (double)(PD - r0) * ll0;
            if (rk < PD) ck += (double)(PD - rk) * llk;
            const double cst = ck - c0;
            const double nuP = lam[k] + ib;
            const double t = rk < PD ? 1.0 / nuP : 0.0;
            const double gP = rk < PD ? lam[k] * t : 0.0;
            red[0] = t;
            red[1] = gP;
            s_ib = ib;
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
            const float inumin = rk < PD ? (float)t : (float)(1.0 / (S[(size_t)k * PD + PD - 1] + ib));
            atomicMax(reinterpret_cast<int *>(tab.tmax), __float_as_int(inumin));
        }
    }
    __syncthreads();
    const double ib = s_ib, t = red[0], gP = red[1];
    __syncthreads();  // red is reused below
    const int o = roff[k], rp = roff[k + 1] - o;
    for (int jj = j; jj < rp; jj += 64) {
        double q = 0.0, gw = 0.0;
        if (jj < rk) {
            const double inu = 1.0 / (S[(size_t)k * PD + jj] + ib);
            q = inu - t;
            gw = S[(size_t)k * PD + jj] * inu - gP;
        }
        float qh = (float)q;
        tab.q_hi[o + jj] = qh;
        tab.q_lo[o + jj] = (float)(q - (double)qh);
        tab.gw[o + jj] = (float)gw;
        const float sv = jj < rk ? sqrtf(fabsf(qh)) : 0.0f;  // basis scale: FP32 suffices
        sq[jj] = sv;
        tab.sq[o + jj] = sv;
    }
    if (!(fmt & 8)) return;
    __syncthreads();
    // per-component scale of the E4M3 basis: the largest |value| maps to 448
    float m = 0.0f;
    for (int jj = 0; jj < rk; ++jj) m = fmaxf(m, fabsf(B[(size_t)j * Rtot + o + jj] * sq[jj]));
    red[j] = m;
    __syncthreads();
    for (int st = 32; st > 0; st >>= 1) {
        if (j < st) red[j] = fmax(red[j], red[j + st]);
        __syncthreads();
    }
    const float s8 = red[0] > 0.0 ? (float)red[0] / 448.0f : 1.0f;
    if (j == 0) {
        tab.k8s2[k] = s8 * s8;
        tab.k8s[k] = s8;
    }
}

// Scaled bases, K-major: Bx[col][e] = 16-bit(U[e][col] * sqrt|q_col|); the
// split form stores the BF16 value and the BF16 remainder; E4M3 divides by
// the component's scale.  B is e-major, so a block transposes a 32-column x
// 64-row tile through shared memory: read along the columns, written along e.
// Grid (Rtot / 32, nb), 256 threads.
__global__ void __launch_bounds__(256)
k_scale_basis(int K, int Rtot, int Rp, const int *__restrict__ colk, const float *__restrict__ B, Tables tab0,
              int fmt)
{
    pdl_enter();
    __shared__ float tile[PD][33];
    const Tables tab = slot_tables(tab0, blockIdx.y, K, Rp, Rtot);
    const int c0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
#pragma unroll
    for (int e = ty; e < PD; e += 8) tile[e][tx] = B[(size_t)e * Rtot + c0 + tx] * tab.sq[c0 + tx];
    __syncthreads();
    // write: column c0 + cl, elements e = 2 tx, 2 tx + 1 (32 threads cover one 64-element row)
#pragma unroll
    for (int cl = ty; cl < 32; cl += 8) {
        const int col = c0 + cl;
        const size_t dst = (size_t)col * PD + 2 * tx;
        const float v0 = tile[2 * tx][cl], v1 = tile[2 * tx + 1][cl];
        const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
        if (fmt & 1) *reinterpret_cast<__nv_bfloat162 *>(tab.B1 + dst) = h;
        if (fmt & 2) *reinterpret_cast<__half2 *>(tab.B1 + dst) = __floats2half2_rn(v0, v1);
        if (fmt & 4) {
            *reinterpret_cast<__nv_bfloat162 *>(tab.Bs + dst) = h;
            *reinterpret_cast<__nv_bfloat162 *>(tab.Bs_lo + dst) =
                __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
        }
        if (fmt & 8) {
            const int k = colk[col];
            const float s8 = k >= 0 && k < K ? tab.k8s[k] : 1.0f;
            tab.B8[dst] = (uint8_t)__nv_cvt_float_to_fp8(v0 / s8, __NV_SATFINITE, __NV_E4M3);
            tab.B8[dst + 1] = (uint8_t)__nv_cvt_float_to_fp8(v1 / s8, __NV_SATFINITE, __NV_E4M3);
        }
    }
}

epll_status launch_tables(epll_gmm *g, const double *d_lambda, const double *mult, int nb,
                          double sigma2, double beta_direct, int fmt, cudaStream_t st)
{
    Mults m{};
    for (int b = 0; b < nb; ++b) m.m[b] = mult[b];
    EPLL_CU(cudaMemsetAsync(g->tab0.tmax, 0, sizeof(float) * nb, st));
    EPLL_CU(launch_pdl(k_tables, dim3(dim3(g->K, nb)), dim3(64), 0, st, g->K, g->Rtot, g->Rp, g->d_r, g->d_roff, g->d_S, g->d_w,
                                            g->d_lam, d_lambda, m, sigma2, beta_direct, g->d_B, g->tab0, fmt));
    EPLL_LAUNCHED(g);
    if (fmt) {
        EPLL_CU(launch_pdl(k_scale_basis, dim3(dim3(g->Rtot / 32, nb)), dim3(256), 0, st, g->K, g->Rtot, g->Rp, g->d_colk, g->d_B, g->tab0,
                                                              fmt));
        EPLL_LAUNCHED(g);
    }
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

// ---------------------------------------------------------------- valid boundary
// Every patch inside the image, raster order: anchor g is (g / nj, g % nj)
// with nj = W - 7.
__global__ void k_valid(int H, int W, int nb, int *__restrict__ anchors_all, unsigned *__restrict__ mult_all)
{
    const int nj = W - PS + 1, n = (H - PS + 1) * nj;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int a = (g / nj) * W + g % nj;
    for (int b = 0; b < nb; ++b) {
        anchors_all[(size_t)b * H * W + g] = a;
        mult_all[(size_t)b * H * W + a] = 1u;
    }
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

// One launch: a thread-block cluster per iteration of the batch (16 CTAs
// where the device allows it, else 8) splits the N anchors into contiguous
// slices.  Each radix pass, every CTA builds the 256-bin histogram of its
// slice's keys that match the threshold determined so far; after a cluster
// barrier every CTA sums all histograms through distributed shared memory (in
// rank order) and takes the same digit.  The compaction then counts, per CTA,
// the keys below / equal to the threshold, exchanges the counts the same way
// (each CTA's base is the sum over lower ranks), and writes its slice's
// selected anchors in anchor order: tiles of 1024 x 8 consecutive anchors,
// each thread eight of them, positions from a block-wide scan.  The keys are
// hashed once when the slice fits in shared memory.
constexpr int FS_THREADS = 1024;

__device__ unsigned long long block_excl_scan_u64(unsigned long long v, unsigned long long &total)
{
    __shared__ unsigned long long ws_[FS_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws_[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long z = ws_[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        ws_[lane] = z;
    }
    __syncthreads();
    const unsigned long long before = (wid ? ws_[wid - 1] : 0ull) + x - v;
    total = ws_[31];
    __syncthreads();
    return before;
}

// Keys of a slice are cached in dynamic shared memory when the slice fits
// (`cached`), else recomputed in every pass.
constexpr int FS_CACHE_BYTES = 160 * 1024;

__global__ void __launch_bounds__(FS_THREADS, 1)
k_frac_cluster(int N, int M, uint64_t seed, int t0, int cached, int *__restrict__ anchors_all,
               unsigned *__restrict__ mult_all)
{
    pdl_enter();
    extern __shared__ uint32_t kc[];
    namespace cgx = cooperative_groups;
    cgx::cluster_group cl = cgx::this_cluster();
    __shared__ unsigned hist[256];
    __shared__ unsigned long long cnt_s;  // (less << 32) | eq of this CTA's slice
    __shared__ unsigned sel[3];           // prefix, mask, rank
    const int nb = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int slot = blockIdx.x / nb;
    const int t = t0 + slot;
    int *anchors = anchors_all + (size_t)slot * N;
    unsigned *mult = mult_all + (size_t)slot * N;
    const uint64_t st = stream_state(seed, (uint64_t)t);
    const int chunk = (N + nb - 1) / nb;
    const int a0 = min(N, rank * chunk), a1 = min(N, a0 + chunk);
    unsigned prefix = 0u, mask = 0u, R = (unsigned)(M - 1);
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        if (threadIdx.x < 256) hist[threadIdx.x] = 0u;
        __syncthreads();
        for (int a = a0 + threadIdx.x; a < a1; a += FS_THREADS) {
            uint32_t key;
            if (cached && pass) {
                key = kc[a - a0];
            } else {
                key = frac_key(st, a);
                if (cached) kc[a - a0] = key;
            }
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        cl.sync();
        unsigned hd = 0u;
        if (threadIdx.x < 256)
            for (int r = 0; r < nb; ++r) hd += cl.map_shared_rank(hist, r)[threadIdx.x];
        unsigned long long tot;
        const unsigned before = (unsigned)block_excl_scan_u64(threadIdx.x < 256 ? hd : 0u, tot);
        if (threadIdx.x < 256 && hd && before <= R && R < before + hd) {
            sel[0] = prefix | ((unsigned)threadIdx.x << shift);
            sel[1] = mask | (255u << shift);
            sel[2] = R - before;
        }
        cl.sync();  // the digit is known and nobody reads the histograms any more
        prefix = sel[0];
        mask = sel[1];
        R = sel[2];
    }
    const uint32_t thr = prefix;
    const unsigned need = R + 1u;  // keys equal to thr that are selected
    // counts of this slice, then the sums over the lower ranks
    unsigned less = 0u, eq = 0u;
    for (int a = a0 + threadIdx.x; a < a1; a += FS_THREADS) {
        const uint32_t key = cached ? kc[a - a0] : frac_key(st, a);
        less += key < thr;
        eq += key == thr;
    }
    unsigned long long tot;
    (void)block_excl_scan_u64(((unsigned long long)less << 32) | eq, tot);
    if (threadIdx.x == 0) cnt_s = tot;
    cl.sync();
    unsigned long long base = 0ull;
    for (int r = 0; r < rank; ++r) base += *cl.map_shared_rank(&cnt_s, r);
    cl.sync();  // no CTA reads another's shared memory after this
    unsigned lb = (unsigned)(base >> 32), eb = (unsigned)(base & 0xffffffffu);
    for (int tb = a0; tb < a1; tb += FS_THREADS * FRAC_ITEMS) {
        const int b = tb + threadIdx.x * FRAC_ITEMS;
        uint32_t keys[FRAC_ITEMS];
        unsigned l = 0u, e = 0u;
#pragma unroll
        for (int q = 0; q < FRAC_ITEMS; ++q) {
            const int a = b + q;
            keys[q] = a < a1 ? (cached ? kc[a - a0] : frac_key(st, a)) : 0xffffffffu;
            if (a < a1) {
                l += keys[q] < thr;
                e += keys[q] == thr;
            }
        }
        unsigned long long ttot;
        const unsigned long long pre = block_excl_scan_u64(((unsigned long long)l << 32) | e, ttot);
        unsigned ml = lb + (unsigned)(pre >> 32), me = eb + (unsigned)(pre & 0xffffffffu);
#pragma unroll
        for (int q = 0; q < FRAC_ITEMS; ++q) {
            const int a = b + q;
            if (a >= a1) break;
            const bool take = keys[q] < thr || (keys[q] == thr && me < need);
            if (take) anchors[ml + (me < need ? me : need)] = a;
            mult[a] = take ? 1u : 0u;
            ml += keys[q] < thr;
            me += keys[q] == thr;
        }
        lb += (unsigned)(ttot >> 32);
        eb += (unsigned)(ttot & 0xffffffffu);
    }
}

// Cluster size of the fraction sampler (16 where one such cluster fits, else 8).
static int frac_cluster_size()
{
    static int size = 0;
    if (size) return size;
    size = 8;
    cudaFuncSetAttribute(k_frac_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, FS_CACHE_BYTES);
    if (cudaFuncSetAttribute(k_frac_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(FS_THREADS);
        cfg.dynamicSmemBytes = FS_CACHE_BYTES;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_frac_cluster, &cfg) == cudaSuccess && nclusters > 0)
            size = 16;
    }
    cudaGetLastError();
    return size;
}

void sampler_setup() { (void)frac_cluster_size(); }

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
    if (o.subset == EPLL_SUBSET_VALID) return (H - PS + 1) * (W - PS + 1);
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
    if (o.subset == EPLL_SUBSET_VALID) {
        EPLL_CU(cudaMemsetAsync(mult, 0, sizeof(unsigned) * (size_t)N * nb, st));
        k_valid<<<(*n + 255) / 256, 256, 0, st>>>(H, W, nb, anchors, mult);
        EPLL_LAUNCHED(g);
        return EPLL_OK;
    }
    if (o.subset == EPLL_SUBSET_JITTER || o.subset == EPLL_SUBSET_REGULAR) {
        const int s = (int)o.subset_param;
        EPLL_CU(cudaMemsetAsync(mult, 0, sizeof(unsigned) * (size_t)N * nb, st));
        const int ni = (H + s - 1) / s, nj = (W + s - 1) / s;
        k_jitter<<<dim3((ni * nj + 255) / 256, nb), 256, 0, st>>>(
            H, W, s, o.seed, t0, ni, nj, o.subset == EPLL_SUBSET_REGULAR ? 1 : 0, anchors, mult);
        EPLL_LAUNCHED(g);
        return EPLL_OK;
    }
    // FRACTION: one cluster per iteration of the batch
    (void)scratch;
    (void)sstride;
    const int cls = frac_cluster_size();
    const size_t slice = ((size_t)N + cls - 1) / cls;
    const int cached = slice * sizeof(uint32_t) <= (size_t)FS_CACHE_BYTES;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cls * nb);
    cfg.blockDim = dim3(FS_THREADS);
    cfg.dynamicSmemBytes = cached ? slice * sizeof(uint32_t) : 0;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cls;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = t_pdl ? 2 : 1;
    EPLL_CU(cudaLaunchKernelEx(&cfg, k_frac_cluster, N, *n, o.seed, t0, cached, anchors, mult));
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

}  // namespace epll
