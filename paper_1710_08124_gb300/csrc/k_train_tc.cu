// Training GEMMs of the proposal network on the tensor cores (tcgen05).
//
// Every forward and backward product of training, C = A B with A(m, k) =
// A[m sam + k sak] and B(k, n) = B[k sbk + n sbn] in FP32 (activations,
// logits' gradients, the BF16-rounded weights), runs as BF16 MMAs with FP32
// accumulation in TMEM.  Each operand is split into a BF16 value and the BF16
// rounding of its remainder, and the three products hi*hi + lo*hi + hi*lo are
// accumulated (the same split form as the selection's exact pass), so the
// gradients keep about 16 bits more than one BF16 product would: close to
// FP32 and within the tolerance the gradient check against the FP64 oracle
// uses.
//
// A CTA computes a 128 x BN tile of C over its share of the reduction: the
// threads read the FP32 operands in 64-deep chunks (coalesced along whichever
// of m / n or k is contiguous), split them and store them in the
// 128-byte-swizzled K-major layout of the MMA operands; two stages let the
// next chunk load while the tensor core multiplies the current one.  Long
// reductions (the weight gradients sum over the batch) are split across CTAs
// (grid z) into partial tiles that a second kernel adds in a fixed order.
#include "epll_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

namespace epll {

constexpr int TG_M = 128;        // rows per CTA (the MMA's M)
constexpr int TG_THREADS = 256;  // eight warps: operand fill, then the epilogue
constexpr int TG_KC = 64;        // reduction chunk: one 128-byte row per operand row

template <int BN>
struct TgCfg {
    static constexpr int A_T = TG_M * 128;
    static constexpr int B_T = BN * 128;
    static constexpr int STAGE = 2 * A_T + 2 * B_T;  // A hi, A lo, B hi, B lo
    static constexpr int TCOLS = BN < 32 ? 32 : BN;  // TMEM columns (a power of two)
    static constexpr int SMEM = 1024 + 2 * STAGE + 128;
};

struct TgArgs {
    int M, N, Kd;
    const float *A;
    long sam, sak;
    const float *B;
    long sbk, sbn;
    float *C;   // C[m * ldc + n] (+ z * cz for split z)
    int ldc;
    int kper;   // reduction length per split (a multiple of TG_KC)
    long cz;
};

// byte offset of element (row r, column k < 64) in a swizzled K-major tile
__device__ __forceinline__ uint32_t tg_off(int r, int k)
{
    return (uint32_t)(r * 128 + ((((k >> 3) ^ (r & 7))) << 4) + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t *>(&v); }

// rows r0.. of a [rows][64] operand chunk: element (r, k) = src[(row0 + r) * sr + (k0 + k) * sk]
// (zero outside rows < nrows, k0 + k < kend), split into hi / lo tiles.
template <int ROWS>
__device__ __forceinline__ void tg_fill(unsigned char *hi, unsigned char *lo, const float *__restrict__ src, long sr,
                                        long sk, int row0, int nrows, int k0, int kend)
{
    // one pair of columns (k, k + 1) per work unit; consecutive threads take
    // consecutive units along the contiguous dimension of the source
    const bool along_k = sk == 1;
#pragma unroll 4
    for (int u = threadIdx.x; u < ROWS * (TG_KC / 2); u += TG_THREADS) {
        int r, kp;
        if (along_k) {
            r = u / (TG_KC / 2);
            kp = u % (TG_KC / 2);
        } else {
            r = u % ROWS;
            kp = u / ROWS;
        }
        const int k = 2 * kp, gr = row0 + r, gk = k0 + k;
        float v0 = 0.0f, v1 = 0.0f;
        if (gr < nrows) {
            if (gk < kend) v0 = src[(long)gr * sr + (long)gk * sk];
            if (gk + 1 < kend) v1 = src[(long)gr * sr + (long)(gk + 1) * sk];
        }
        const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
        const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
        const uint32_t o = tg_off(r, k);
        *reinterpret_cast<uint32_t *>(hi + o) = bf16x2_bits(h);
        *reinterpret_cast<uint32_t *>(lo + o) = bf16x2_bits(l);
    }
}

template <int BN>
__global__ void __launch_bounds__(TG_THREADS, 1) k_gemm_tc(TgArgs g, int *__restrict__ err)
{
    using C = TgCfg<BN>;
    extern __shared__ __align__(1024) unsigned char tg_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)tg_raw + 1023) & ~(uintptr_t)1023);
    unsigned long long *done = reinterpret_cast<unsigned long long *>(smem + 2 * C::STAGE);  // per stage
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * TG_M, n0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * g.kper, kend = min(g.Kd, kbeg + g.kper);
    const int nchunks = kend > kbeg ? (kend - kbeg + TG_KC - 1) / TG_KC : 0;
    float *Cz = g.C + (long)blockIdx.z * g.cz;
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        mbar_init(smem_u32(&done[0]), 1);
        mbar_init(smem_u32(&done[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "n"(C::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t idesc = idesc_f16(TG_M, BN, 1);
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        unsigned char *Ahi = smem + s * C::STAGE, *Alo = Ahi + C::A_T, *Bhi = Alo + C::A_T, *Blo = Bhi + C::B_T;
        // the stage's previous MMAs (chunk c - 2) are complete before it is refilled
        if (c >= 2) ok = ok && mbar_wait(smem_u32(&done[s]), ((c - 2) >> 1) & 1, abort_flag);
        const int k0 = kbeg + c * TG_KC;
        tg_fill<TG_M>(Ahi, Alo, g.A, g.sam, g.sak, m0, g.M, k0, kend);
        tg_fill<BN>(Bhi, Blo, g.B, g.sbn, g.sbk, n0, g.N, k0, kend);
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0 && ok) {
            tc_fence_after();
            const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
            for (int kk = 0; kk < TG_KC / 16; ++kk) {
                const uint32_t q = 32 * kk;
                mma_f16(tbase, sdesc_sw128(ah + q), sdesc_sw128(bh + q), idesc, (c > 0 || kk > 0) ? 1u : 0u);
                mma_f16(tbase, sdesc_sw128(al + q), sdesc_sw128(bh + q), idesc, 1u);
                mma_f16(tbase, sdesc_sw128(ah + q), sdesc_sw128(bl + q), idesc, 1u);
            }
            mma_commit(smem_u32(&done[s]));
        }
    }
    // the last commit tracks every MMA issued before it
    if (nchunks > 0) {
        const int c = nchunks - 1;
        ok = ok && mbar_wait(smem_u32(&done[c & 1]), (c >> 1) & 1, abort_flag);
    }
    __syncwarp();
    ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
    tc_fence_after();
    // epilogue: warp w reads TMEM lane quarter w % 4 (rows 32 (w % 4) ..) and
    // half w / 4 of the columns, 32 at a time
    const int q4 = warp & 3, hh = warp >> 2;
    const int row = 32 * q4 + lane, gm = m0 + row;
    for (int cb = hh * (BN / 2); cb < (hh + 1) * (BN / 2); cb += 32) {
        uint32_t v[32];
        if (ok && nchunks > 0) {
            tmem_ld_all<32>(tbase + ((uint32_t)(32 * q4) << 16) + (uint32_t)cb, v);
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = 0u;
        }
        if (gm < g.M) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int gn = n0 + cb + j;
                if (gn < g.N) Cz[(long)gm * g.ldc + gn] = __uint_as_float(v[j]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(C::TCOLS) : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(err, 1);
}

// out[m][n] = sum over z of part[z][m][n], in increasing z
__global__ void k_splitk_sum(const float *__restrict__ part, int splits, int M, int N, long cz, float *__restrict__ out,
                             int ldc)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)M * N) return;
    const int m = (int)(i / N), n = (int)(i % N);
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += part[(long)z * cz + (long)m * N + n];
    out[(long)m * ldc + n] = s;
}

template <int BN>
static epll_status launch_gemm_tc(const TgArgs &a, dim3 grid, int *err, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        EPLL_CU(cudaFuncSetAttribute(k_gemm_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, TgCfg<BN>::SMEM));
        attr = true;
    }
    k_gemm_tc<BN><<<grid, TG_THREADS, TgCfg<BN>::SMEM, st>>>(a, err);
    EPLL_CU(cudaGetLastError());
    return EPLL_OK;
}

epll_status gemm_tc(const float *A, long sam, long sak, const float *B, long sbk, long sbn, float *C, int ldc, int M,
                    int N, int Kd, float *partial, size_t partial_cap, int *err, cudaStream_t st)
{
    const int BN = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
    if (N > 256) return fail(EPLL_EUNSUPPORTED, "training GEMM: N above 256");
    const int mt = (M + TG_M - 1) / TG_M, nt = (N + BN - 1) / BN;
    // split long reductions so that about one CTA per SM works
    int splits = 1;
    if (mt * nt < 64 && Kd >= 8 * TG_KC) {
        splits = 148 / (mt * nt);
        const int maxs = Kd / (4 * TG_KC);
        if (splits > maxs) splits = maxs;
        if (splits < 1) splits = 1;
        while (splits > 1 && (size_t)splits * M * N > partial_cap) --splits;
    }
    int kper = (Kd + splits - 1) / splits;
    kper = (kper + TG_KC - 1) / TG_KC * TG_KC;
    splits = (Kd + kper - 1) / kper;
    TgArgs a{M, N, Kd, A, sam, sak, B, sbk, sbn, C, ldc, kper, 0};
    if (splits > 1) {
        a.C = partial;
        a.ldc = N;
        a.cz = (long)M * N;
    }
    const dim3 grid(mt, nt, splits);
    epll_status s;
    if (BN == 64) s = launch_gemm_tc<64>(a, grid, err, st);
    else if (BN == 128) s = launch_gemm_tc<128>(a, grid, err, st);
    else s = launch_gemm_tc<256>(a, grid, err, st);
    if (s) return s;
    if (splits > 1) {
        const long tot = (long)M * N;
        k_splitk_sum<<<(int)((tot + 255) / 256), 256, 0, st>>>(partial, splits, M, N, (long)M * N, C, ldc);
        EPLL_CU(cudaGetLastError());
    }
    return EPLL_OK;
}

}  // namespace epll
