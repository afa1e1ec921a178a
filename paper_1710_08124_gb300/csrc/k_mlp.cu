// Learned top-m proposal for the Gaussian selection.
//
// A small network, 64 -> 256 -> 256 -> K with GELU, maps a DC-free patch
// (scaled by sqrt(beta), with log(1/beta) entering the first layer through a
// learned per-unit coefficient, so that the selection label of Eq. 14 is a
// function of the input) to logits over the K components.  Inference runs on
// the tensor cores (one tcgen05 kernel per layer, BF16 operands, FP32
// accumulation in TMEM, bias + GELU or bias + top-m fused in the epilogue).
// The m proposed components of every patch are rescored exactly in FP32 --
// the (patch, candidate) pairs grouped by component, each group's basis in
// shared memory -- and a patch whose proposals carry too little softmax mass
// or whose rescored top-2 gap is within the FP32 error bound goes to the
// exhaustive split-BF16 pass (and, if still undecided, to the compensated
// rescoring): exhaustive scoring is both the fallback and the judge.
//
// Training (BF16-rounded weights, FP32 activations and accumulation, FP32
// master weights, AdamW) runs its products on the tensor cores in the split
// BF16 form (k_train_tc.cu) and the elementwise steps in SIMT FP32; it runs
// offline on (patch, exact selection) pairs produced by the exhaustive path.
#include "epll_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

namespace epll {

constexpr int HID = 256;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + HID * PD;
constexpr int OFF_WB = OFF_B1 + HID;
constexpr int OFF_W2 = OFF_WB + HID;
constexpr int OFF_B2 = OFF_W2 + HID * HID;
constexpr int OFF_W3 = OFF_B2 + HID;
__host__ __device__ inline size_t off_b3(int K) { return (size_t)OFF_W3 + (size_t)HID * K; }
__host__ __device__ inline size_t prop_size(int K) { return off_b3(K) + (size_t)K; }

}  // namespace epll

struct epll_proposal {
    int K = 0;
    size_t np = 0;
    float *theta = nullptr, *mom1 = nullptr, *mom2 = nullptr, *grad = nullptr;
    float *wr = nullptr;  // theta with W1, W2, W3 rounded to BF16 (the weights every forward uses)
    uint16_t *W1b = nullptr, *W2b = nullptr, *W3b = nullptr;  // BF16 [256][64], [256][256], [256][256]
    long long step = 0;
    int Bmax = 0;
    float *X = nullptr, *cond = nullptr, *A1 = nullptr, *H1 = nullptr, *A2 = nullptr, *H2 = nullptr;
    float *L = nullptr, *dH = nullptr, *dA = nullptr, *loss = nullptr;
    float *partial = nullptr;  // split-K partial products
};

namespace epll {

// GELU in its tanh form: 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).
constexpr float GELU_A = 0.7978845608028654f, GELU_B = 0.044715f;
__device__ __forceinline__ float gelu_f(float x)
{
    return 0.5f * x * (1.0f + tanhf(GELU_A * fmaf(GELU_B * x, x * x, x)));
}
__device__ __forceinline__ float gelu_grad_f(float x)
{
    const float t = tanhf(GELU_A * fmaf(GELU_B * x, x * x, x));
    return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * GELU_A * fmaf(3.0f * GELU_B, x * x, 1.0f);
}
// Inference form: the hardware tanh approximation (about 11 correct bits,
// below the BF16 rounding that follows).
__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float gelu_fast(float x)
{
    const float hx = 0.5f * x;
    return fmaf(hx, tanh_fast(GELU_A * fmaf(GELU_B * x, x * x, x)), hx);
}

// ============================================================================
// Training kernels: the products run on the tensor cores (k_train_tc.cu); the
// elementwise steps (gather, bias + GELU, softmax cross-entropy, GELU
// derivative, column sums, AdamW, BF16 rounding) are SIMT FP32.
// ============================================================================
// X[b] = (patch - mean) * exp(-log_ib/2), cond[b] = log_ib; one warp per sample
__global__ void k_mlp_gather(const float *__restrict__ images, int n_img, int H, int W,
                             const int *__restrict__ img_idx, const int *__restrict__ anchors,
                             const float *__restrict__ log_ib, const int *__restrict__ sel, int n_all, int B,
                             float *__restrict__ X, float *__restrict__ cond, int *__restrict__ bad)
{
    const int b = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (b >= B) return;
    const int s = sel ? sel[b] : b;
    const bool ok_s = s >= 0 && s < n_all;
    const int im_i = ok_s ? img_idx[s] : -1;
    const int a = ok_s ? anchors[s] : -1;
    const float lib = ok_s ? log_ib[s] : 0.0f;
    if (!ok_s || im_i < 0 || im_i >= n_img || a < 0 || a >= H * W || !isfinite(lib)) {
        if (lane == 0) {
            atomicExch(bad, 1);
            cond[b] = 0.0f;
        }
        X[(size_t)b * PD + lane] = 0.0f;
        X[(size_t)b * PD + lane + 32] = 0.0f;
        return;
    }
    const float *im = images + (size_t)im_i * H * W;
    const int ai = a / W, aj = a % W;
    int r0 = ai + (lane >> 3), r1 = r0 + 4, c = aj + (lane & 7);
    if (r0 >= H) r0 -= H;
    if (r1 >= H) r1 -= H;
    if (c >= W) c -= W;
    const float x0 = im[(size_t)r0 * W + c], x1 = im[(size_t)r1 * W + c];
    float sum = x0 + x1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const float mu = sum * (1.0f / PD), sc = expf(-0.5f * lib);
    X[(size_t)b * PD + lane] = (x0 - mu) * sc;
    X[(size_t)b * PD + lane + 32] = (x1 - mu) * sc;
    if (lane == 0) cond[b] = lib;
}

// A += bias (+ cond * wb) in place; Hout = gelu(A)
__global__ void k_bias_gelu(float *__restrict__ A, const float *__restrict__ bias, const float *__restrict__ wb,
                            const float *__restrict__ cond, int B, float *__restrict__ Hout)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)B * HID) return;
    const int j = (int)(i % HID), b = (int)(i / HID);
    const float v = A[i] + bias[j] + (wb ? cond[b] * wb[j] : 0.0f);
    A[i] = v;
    Hout[i] = gelu_f(v);
}

// logits += b3; dL = (softmax - onehot) / B; loss += mean cross-entropy.
// One warp per sample (lanes over the components), the block's loss terms
// summed before one atomic per block.
constexpr int SM_WARPS = 8;
__global__ void __launch_bounds__(32 * SM_WARPS)
k_softmax_ce(float *__restrict__ Lg, const float *__restrict__ b3, const int *__restrict__ labels,
             const int *__restrict__ sel, int n_all, int B, int K, float *__restrict__ loss, int *__restrict__ bad)
{
    __shared__ float part[SM_WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * SM_WARPS + warp;
    float term = 0.0f;
    if (b < B) {
        const int s = sel ? sel[b] : b;
        const int lab = (s >= 0 && s < n_all) ? labels[s] : -1;
        float *l = Lg + (size_t)b * K;
        if (lab < 0 || lab >= K) {  // invalid label: no gradient from this sample
            if (lane == 0) atomicExch(bad, 1);
            for (int k = lane; k < K; k += 32) l[k] = 0.0f;
        } else {
            float mx = -FLT_MAX;
            for (int k = lane; k < K; k += 32) {
                const float v = l[k] + b3[k];
                l[k] = v;
                mx = fmaxf(mx, v);
            }
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            float se = 0.0f;
            for (int k = lane; k < K; k += 32) se += expf(l[k] - mx);
            for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
            const float lse = mx + logf(se);
            __syncwarp();
            if (lane == 0) term = (lse - l[lab]) / (float)B;
            __syncwarp();
            for (int k = lane; k < K; k += 32) l[k] = (expf(l[k] - lse) - (k == lab ? 1.0f : 0.0f)) / (float)B;
        }
    }
    if (lane == 0) part[warp] = term;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < SM_WARPS; ++w) t += part[w];
        atomicAdd(loss, t);
    }
}

__global__ void k_gelu_back(float *__restrict__ dH, const float *__restrict__ A, long n)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dH[i] *= gelu_grad_f(A[i]);
}

// out[n] = sum_b D[b][n] (optionally weighted by cond[b]).  Block (32 x 32):
// thread (x, y) sums the rows b = y (mod 32) of column 32 blockIdx.x + x in
// increasing b, then the 32 partial sums of a column are added in order of y.
__global__ void __launch_bounds__(1024) k_colsum(const float *__restrict__ D, int B, int N,
                                                 const float *__restrict__ cond, float *__restrict__ out)
{
    __shared__ float ps[32][33];
    const int n = blockIdx.x * 32 + threadIdx.x;
    float s = 0.0f;
    if (n < N)
        for (int b = threadIdx.y; b < B; b += 32) s = fmaf(cond ? cond[b] : 1.0f, D[(size_t)b * N + n], s);
    ps[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && n < N) {
        float t = 0.0f;
        for (int y = 0; y < 32; ++y) t += ps[y][threadIdx.x];
        out[n] = t;
    }
}

// AdamW (decoupled weight decay on the weight matrices only), then the BF16
// roundings of the weights (training forward and inference copies).
__global__ void k_adamw(float *__restrict__ th, const float *__restrict__ g, float *__restrict__ m1,
                        float *__restrict__ m2, long np, int K, float lr, float wd, float c1, float c2)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const bool is_w = i < OFF_B1 || (i >= OFF_W2 && i < OFF_B2) || (i >= OFF_W3 && i < (long)off_b3(K));
    const float gi = g[i];
    const float a = 0.9f * m1[i] + 0.1f * gi, b = 0.999f * m2[i] + 0.001f * gi * gi;
    m1[i] = a;
    m2[i] = b;
    float t = th[i];
    if (is_w) t -= lr * wd * t;
    th[i] = t - lr * (a / c1) / (sqrtf(b / c2) + 1e-8f);
}

__global__ void k_round_weights(const float *__restrict__ th, long np, int K, float *__restrict__ wr,
                                uint16_t *__restrict__ W1b, uint16_t *__restrict__ W2b, uint16_t *__restrict__ W3b)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const bool is_w = i < OFF_B1 || (i >= OFF_W2 && i < OFF_B2) || (i >= OFF_W3 && i < (long)off_b3(K));
    const __nv_bfloat16 h = __float2bfloat16_rn(th[i]);
    wr[i] = is_w ? __bfloat162float(h) : th[i];
    if (i < OFF_B1) W1b[i] = __bfloat16_as_ushort(h);
    else if (i >= OFF_W2 && i < OFF_B2) W2b[i - OFF_W2] = __bfloat16_as_ushort(h);
    else if (i >= OFF_W3 && i < (long)off_b3(K)) W3b[i - OFF_W3] = __bfloat16_as_ushort(h);
}

// split-K partial tiles of the training products (up to 74 splits of a 256 x 256 result)
constexpr size_t TRAIN_PARTIAL = (size_t)74 * HID * HID;

static epll_status gemm(epll_proposal *p, const float *A, long sam, long sak, const float *B, long sbk, long sbn,
                        float *C, int ldc, int M, int N, int Kd, cudaStream_t st)
{
    return gemm_tc(A, sam, sak, B, sbk, sbn, C, ldc, M, N, Kd, p->partial, TRAIN_PARTIAL,
                   reinterpret_cast<int *>(p->loss + 2), st);
}

static epll_status ensure_train(epll_proposal *p, int B)
{
    if (B <= p->Bmax) return EPLL_OK;
    float *ptrs[] = {p->X, p->cond, p->A1, p->H1, p->A2, p->H2, p->L, p->dH, p->dA, p->partial};
    for (float *q : ptrs)
        if (q) cudaFree(q);
    const size_t HB = (size_t)B * HID;
    cudaError_t e = cudaSuccess;
    auto A = [&](float **q, size_t n) { if (e == cudaSuccess) e = cudaMalloc(q, sizeof(float) * n); };
    A(&p->X, (size_t)B * PD); A(&p->cond, B); A(&p->A1, HB); A(&p->H1, HB); A(&p->A2, HB); A(&p->H2, HB);
    A(&p->L, (size_t)B * p->K); A(&p->dH, HB > (size_t)B * p->K ? HB : (size_t)B * p->K); A(&p->dA, HB);
    A(&p->partial, TRAIN_PARTIAL);
    if (e != cudaSuccess) {
        p->Bmax = 0;
        return fail(EPLL_ENOMEM, std::string("proposal training buffers: ") + cudaGetErrorString(e));
    }
    p->Bmax = B;
    return EPLL_OK;
}

// Forward + backward of the mean cross-entropy on one batch; gradient in p->grad.
struct Batch {
    const float *images;
    int n_img, H, W;
    const int *img_idx, *anchors;
    const float *log_ib;
    const int *labels, *sel;
    int n_all, B;
};

static epll_status forward_backward(epll_proposal *p, const Batch &d, cudaStream_t st)
{
    epll_status s;
    const int B = d.B;
    if ((s = ensure_train(p, B))) return s;
    const int K = p->K;
    int *bad = reinterpret_cast<int *>(p->loss + 1);
    const float *w = p->wr;
    float *g = p->grad;
    EPLL_CU(cudaMemsetAsync(p->loss, 0, 3 * sizeof(float), st));
    k_mlp_gather<<<(B + 3) / 4, 128, 0, st>>>(d.images, d.n_img, d.H, d.W, d.img_idx, d.anchors, d.log_ib, d.sel,
                                              d.n_all, B, p->X, p->cond, bad);
    EPLL_CU(cudaGetLastError());
    const long HB = (long)B * HID;
    const int eb = (int)((HB + 255) / 256);
    // forward
    if ((s = gemm(p, p->X, PD, 1, w + OFF_W1, 1, PD, p->A1, HID, B, HID, PD, st))) return s;
    k_bias_gelu<<<eb, 256, 0, st>>>(p->A1, w + OFF_B1, w + OFF_WB, p->cond, B, p->H1);
    if ((s = gemm(p, p->H1, HID, 1, w + OFF_W2, 1, HID, p->A2, HID, B, HID, HID, st))) return s;
    k_bias_gelu<<<eb, 256, 0, st>>>(p->A2, w + OFF_B2, nullptr, nullptr, B, p->H2);
    if ((s = gemm(p, p->H2, HID, 1, w + OFF_W3, 1, HID, p->L, K, B, K, HID, st))) return s;
    k_softmax_ce<<<(B + SM_WARPS - 1) / SM_WARPS, 32 * SM_WARPS, 0, st>>>(p->L, w + off_b3(K), d.labels, d.sel, d.n_all, B, K, p->loss,
                                                  bad);
    EPLL_CU(cudaGetLastError());
    // backward (p->L now holds dL)
    if ((s = gemm(p, p->L, 1, K, p->H2, HID, 1, g + OFF_W3, HID, K, HID, B, st))) return s;    // dW3 = dL^T H2
    k_colsum<<<(K + 31) / 32, dim3(32, 32), 0, st>>>(p->L, B, K, nullptr, g + off_b3(K));
    if ((s = gemm(p, p->L, K, 1, w + OFF_W3, HID, 1, p->dH, HID, B, HID, K, st))) return s;    // dH2 = dL W3
    k_gelu_back<<<eb, 256, 0, st>>>(p->dH, p->A2, HB);                                      // dA2
    if ((s = gemm(p, p->dH, 1, HID, p->H1, HID, 1, g + OFF_W2, HID, HID, HID, B, st))) return s;  // dW2
    k_colsum<<<(HID + 31) / 32, dim3(32, 32), 0, st>>>(p->dH, B, HID, nullptr, g + OFF_B2);
    if ((s = gemm(p, p->dH, HID, 1, w + OFF_W2, HID, 1, p->dA, HID, B, HID, HID, st))) return s;  // dH1
    k_gelu_back<<<eb, 256, 0, st>>>(p->dA, p->A1, HB);                                         // dA1
    if ((s = gemm(p, p->dA, 1, HID, p->X, PD, 1, g + OFF_W1, PD, HID, PD, B, st))) return s;     // dW1
    k_colsum<<<(HID + 31) / 32, dim3(32, 32), 0, st>>>(p->dA, B, HID, nullptr, g + OFF_B1);
    k_colsum<<<(HID + 31) / 32, dim3(32, 32), 0, st>>>(p->dA, B, HID, p->cond, g + OFF_WB);
    EPLL_CU(cudaGetLastError());
    return EPLL_OK;
}

static epll_status refresh(epll_proposal *p, cudaStream_t st)
{
    k_round_weights<<<(int)((p->np + 255) / 256), 256, 0, st>>>(p->theta, (long)p->np, p->K, p->wr, p->W1b,
                                                                 p->W2b, p->W3b);
    EPLL_CU(cudaGetLastError());
    return EPLL_OK;
}

// ============================================================================
// Inference: the three layers fused in one persistent tcgen05 kernel.  A CTA
// takes 128-patch tiles in turn; the hidden activations never leave the SM:
//   warp 0      TMA: the tile's BF16 patches (double buffer) and the weight
//               matrices as nine 64-wide K chunks (W1; W2 x4; W3 x4) through a
//               three-slot ring (the weights stay in L2 across tiles);
//   warp 1      MMA: layer l accumulates 128 x 256 FP32 in TMEM (layers 1, 3 at
//               columns 0..255, layer 2 at 256..511), K chunk by K chunk as the
//               epilogue releases the operand chunks;
//   warps 2..   epilogue, one thread per row and a slice of columns per warp:
//               layer 1: v = sqrt(beta) acc + b1 + log(1/beta) wb, layer 2:
//               v = acc + b2, both GELU'd, rounded to BF16 and written to shared
//               memory in the 128-byte-swizzled K-major layout of the next MMA's
//               A operand (chunk c is released to the MMA as soon as it is
//               written, so layer 2's products overlap layer 1's epilogue);
//               layer 3: logits + b3, each warp's top-m and online softmax
//               sums, merged across the warps of a row.
// Every wait is bounded (an abort flag ends all roles; err is raised).
// ============================================================================
constexpr int MT = 128;
constexpr int TOPM_MAX = 8;
constexpr int FM_S = 3;               // weight ring slots
constexpr int FM_SLOT = HID * 128;    // 32 KB: [256 rows][64] BF16
constexpr int FM_ZT = MT * 128;       // 16 KB: [128 rows][64] BF16
constexpr int FM_H = 4 * FM_ZT;       // 64 KB: [128][256] BF16 as four K chunks

template <int EW>
struct FmCfg {
    static constexpr int THREADS = 32 * (2 + EW);
    static constexpr int CG = EW / 4;   // column groups per TMEM lane quarter (16 columns of each chunk)
    static_assert(EW == 16, "the epilogue slices every 64-column chunk into four 16-column groups");
    static constexpr int OFF_H = FM_S * FM_SLOT;
    static constexpr int OFF_Z = OFF_H + FM_H;
    static constexpr int OFF_BIAS = OFF_Z + 2 * FM_ZT;
    static constexpr int OFF_BAR = OFF_BIAS + 4 * HID * 4;
    // full[S], empty[S], zfull[2], zempty[2], hready[4], accfull[3], accfree, mready, mdone
    static constexpr int NBAR = 2 * FM_S + 4 + 4 + 3 + 3;
    static constexpr int SMEM = 1024 + OFF_BAR + NBAR * 8 + 16;
    static_assert(CG * MT * (2 * TOPM_MAX + 2) * 4 <= FM_H, "merge scratch must fit in the activation buffer");
};

// 16 accumulator columns at taddr and at taddr + 64 (this warp's slices of
// two consecutive 64-column K chunks), one wait for both loads.
static __device__ __forceinline__ void tmem_ld_2x16(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : EPLL_R8(0), EPLL_R8(8)
                 : "r"(taddr));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : EPLL_R8(16), EPLL_R8(24)
                 : "r"(taddr + 64u));
    tmem_wait(r);
}


// (v, i) ranks before (w, j): larger logit first, lower index on equal logits
static __device__ __forceinline__ bool before(float v, int i, float w, int j) { return v > w || (v == w && i < j); }

template <int TM>
static __device__ __forceinline__ void topm_insert(float (&tv)[TM], int (&ti)[TM], float v, int i)
{
    if (!before(v, i, tv[TM - 1], ti[TM - 1])) return;
#pragma unroll
    for (int q = 0; q < TM; ++q) {
        if (before(v, i, tv[q], ti[q])) {
            const float t1 = tv[q];
            const int t2 = ti[q];
            tv[q] = v;
            ti[q] = i;
            v = t1;
            i = t2;
        }
    }
}

// One chunk of a hidden layer's epilogue: v = scale * acc + bias, GELU, BF16,
// into chunk c of the activation buffer (swizzled like a TMA SWIZZLE_128B
// load, so the next layer's MMA reads it as its A operand).  acc holds this
// warp's 16 columns 64 c + 16 j .. of its row.
static __device__ __forceinline__ void epi_hidden(const uint32_t *acc, int c, int j, int rit, float scale,
                                                  const float *__restrict__ bias, unsigned char *H)
{
    const int col0 = 64 * c + 16 * j;
    uint32_t packed[8];
#pragma unroll
    for (int q = 0; q < 16; q += 4) {
        const float4 b = *reinterpret_cast<const float4 *>(bias + col0 + q);
        const __nv_bfloat162 p0 = __floats2bfloat162_rn(gelu_fast(fmaf(__uint_as_float(acc[q]), scale, b.x)),
                                                        gelu_fast(fmaf(__uint_as_float(acc[q + 1]), scale, b.y)));
        const __nv_bfloat162 p1 = __floats2bfloat162_rn(gelu_fast(fmaf(__uint_as_float(acc[q + 2]), scale, b.z)),
                                                        gelu_fast(fmaf(__uint_as_float(acc[q + 3]), scale, b.w)));
        packed[q / 2] = *reinterpret_cast<const uint32_t *>(&p0);
        packed[q / 2 + 1] = *reinterpret_cast<const uint32_t *>(&p1);
    }
    unsigned char *rowp = H + c * FM_ZT + rit * 128;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int lc = 2 * j + q;  // logical 16-byte chunk of the 128-byte row
        *reinterpret_cast<uint4 *>(rowp + ((lc ^ (rit & 7)) << 4)) =
            make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
    }
}

template <int EW, int TM>
__global__ void __launch_bounds__(32 * (2 + EW), 1)
k_mlp_fused(const __grid_constant__ CUtensorMap mapZ, const __grid_constant__ CUtensorMap mapW1,
            const __grid_constant__ CUtensorMap mapW2, const __grid_constant__ CUtensorMap mapW3, int n, int K,
            int n3, const float *__restrict__ wr, const float *__restrict__ ibeta, int topm,
            int *__restrict__ cand, float *__restrict__ pmass, int *__restrict__ err)
{
    using C = FmCfg<EW>;
    extern __shared__ __align__(1024) unsigned char fm_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)fm_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *ring = smem, *Hb = smem + C::OFF_H, *Zb = smem + C::OFF_Z;
    float *sb1 = reinterpret_cast<float *>(smem + C::OFF_BIAS), *sb2 = sb1 + HID, *sb3 = sb2 + HID;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + C::OFF_BAR);
    unsigned long long *full = bars, *empty = bars + FM_S, *zfull = bars + 2 * FM_S, *zempty = zfull + 2,
                       *hready = zempty + 2, *accfull = hready + 4, *accfree = accfull + 3,
                       *mready = accfree + 1, *mdone = mready + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + C::NBAR);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = (n + MT - 1) / MT;

    // first layer: W1 (sqrt(beta) z) + b1 + log(1/beta) wb = sqrt(beta) (W1 z) + b1'
    const float ib = ibeta ? *ibeta : 1.0f;
    const float in_scale = ibeta ? 1.0f / sqrtf(ib) : 1.0f, cond = ibeta ? logf(ib) : 0.0f;
    for (int i = threadIdx.x; i < HID; i += blockDim.x) {
        sb1[i] = fmaf(cond, wr[OFF_WB + i], wr[OFF_B1 + i]);
        sb2[i] = wr[OFF_B2 + i];
        sb3[i] = i < K ? wr[off_b3(K) + i] : 0.0f;
    }
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        for (int s = 0; s < FM_S; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&zfull[s]), 1);
            mbar_init(smem_u32(&zempty[s]), 1);
        }
        for (int c = 0; c < 4; ++c) mbar_init(smem_u32(&hready[c]), EW);
        for (int a = 0; a < 3; ++a) mbar_init(smem_u32(&accfull[a]), 1);
        mbar_init(smem_u32(accfree), EW);
        mbar_init(smem_u32(mready), EW);  // every epilogue warp wrote its partial top-m
        mbar_init(smem_u32(mdone), 4);    // the merging warps (one per lane quarter) read them
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            tma_prefetch_desc(&mapZ);
            tma_prefetch_desc(&mapW1);
            tma_prefetch_desc(&mapW2);
            tma_prefetch_desc(&mapW3);
            int L = 0, it = 0;
            for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x, ++it) {
                const int zb = it & 1, zph = (it >> 1) & 1;
                if (!mbar_wait(smem_u32(&zempty[zb]), zph ^ 1, abort_flag)) break;
                mbar_expect_tx(smem_u32(&zfull[zb]), FM_ZT);
                tma_load_2d(smem_u32(Zb + zb * FM_ZT), &mapZ, 0, tile * MT, smem_u32(&zfull[zb]));
                for (int q = 0; q < 9; ++q, ++L) {
                    const int slot = L % FM_S, ph = (L / FM_S) & 1;
                    if (!mbar_wait(smem_u32(&empty[slot]), ph ^ 1, abort_flag)) break;
                    const CUtensorMap *m = q == 0 ? &mapW1 : (q < 5 ? &mapW2 : &mapW3);
                    const int x = q == 0 ? 0 : 64 * ((q - 1) & 3);
                    mbar_expect_tx(smem_u32(&full[slot]), (q < 5 ? HID : n3) * 128);
                    tma_load_2d(smem_u32(ring + slot * FM_SLOT), m, x, 0, smem_u32(&full[slot]));
                }
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t id256 = idesc_f16(MT, HID, 1), id3 = idesc_f16(MT, n3, 1);
            int L = 0, it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
                const int zb = it & 1, zph = (it >> 1) & 1;
                if (it > 0) ok = mbar_wait(smem_u32(accfree), (it - 1) & 1, abort_flag);
                ok = ok && mbar_wait(smem_u32(&zfull[zb]), zph, abort_flag);
                for (int layer = 0; layer < 3 && ok; ++layer) {
                    const uint32_t dcol = layer == 1 ? 256u : 0u;
                    const uint32_t idesc = layer == 2 ? id3 : id256;
                    const int nchunks = layer == 0 ? 1 : 4;
                    for (int c = 0; c < nchunks && ok; ++c, ++L) {
                        const int slot = L % FM_S, ph = (L / FM_S) & 1;
                        ok = mbar_wait(smem_u32(&full[slot]), ph, abort_flag);
                        if (ok && layer > 0) ok = mbar_wait(smem_u32(&hready[c]), layer - 1, abort_flag);
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t a0 = layer == 0 ? smem_u32(Zb + zb * FM_ZT) : smem_u32(Hb + c * FM_ZT);
                        const uint32_t b0 = smem_u32(ring + slot * FM_SLOT);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            mma_f16(tbase + dcol, sdesc_sw128(a0 + 32 * k), sdesc_sw128(b0 + 32 * k), idesc,
                                    (c | k) ? 1u : 0u);
                        mma_commit(smem_u32(&empty[slot]));
                    }
                    if (!ok) break;
                    if (layer == 0) mma_commit(smem_u32(&zempty[zb]));
                    mma_commit(smem_u32(&accfull[layer]));
                }
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int e = warp - 2, qd = warp & 3, j = e >> 2;
        const int rit = 32 * qd + lane;
        const uint32_t tl = tbase + ((uint32_t)(32 * qd) << 16) + (uint32_t)(16 * j);
        float *scratch = reinterpret_cast<float *>(Hb);  // [CG][2 TM + 2][128]
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int row = tile * MT + rit;
            // hidden layers: one TMEM round trip for the warp's four slices,
            // then chunk by chunk into the activation buffer
            bool ok = true;
            for (int layer = 0; layer < 2 && ok; ++layer) {
                // tcgen05.ld is warp-collective: every lane takes the same branch
                ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&accfull[layer]), it & 1, abort_flag));
                if (!ok) break;
                tc_fence_after();
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                    uint32_t acc[32];
                    tmem_ld_2x16(tl + (layer ? 256u : 0u) + 128u * h, acc);
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        const int c = 2 * h + cc;
                        epi_hidden(acc + 16 * cc, c, j, rit, layer ? 1.0f : in_scale, layer ? sb2 : sb1, Hb);
                        fence_proxy_async();
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(smem_u32(&hready[c]));
                    }
                }
            }
            if (ok) ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&accfull[2]), it & 1, abort_flag));
            if (!ok) break;
            tc_fence_after();
            // output layer: this warp's columns 64 c + 16 j + q (increasing in
            // (c, q)), two chunks per TMEM round trip; online softmax sums and
            // top-m without data-dependent branches
            float tv[TM];
            int ti[TM];
#pragma unroll
            for (int q = 0; q < TM; ++q) {
                tv[q] = -FLT_MAX;
                ti[q] = 0x7fffffff;
            }
            float mx = -INFINITY, se = 0.0f;
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                if (128 * h + 16 * j >= K) break;
                uint32_t acc[32];
                tmem_ld_2x16(tl + 128u * h, acc);
                float hm = -INFINITY;
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int col = 128 * h + 64 * (q >> 4) + 16 * j + (q & 15);
                    const float v = col < K ? __uint_as_float(acc[q]) + sb3[col] : -INFINITY;
                    acc[q] = __float_as_uint(v);
                    hm = fmaxf(hm, v);
                }
                const float nm = fmaxf(mx, hm);
                float hs = 0.0f;
                if (nm > -INFINITY) {
#pragma unroll
                    for (int q = 0; q < 32; ++q) hs += __expf(__uint_as_float(acc[q]) - nm);
                }
                se = (mx > -INFINITY ? se * __expf(mx - nm) : 0.0f) + hs;
                mx = nm;
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    // insertion by selects; a tie never displaces (columns ascend)
                    float v = __uint_as_float(acc[q]);
                    int ix = 128 * h + 64 * (q >> 4) + 16 * j + (q & 15);
#pragma unroll
                    for (int u = 0; u < TM; ++u) {
                        const bool sw = v > tv[u];
                        const float tvu = tv[u];
                        const int tiu = ti[u];
                        tv[u] = sw ? v : tvu;
                        ti[u] = sw ? ix : tiu;
                        v = sw ? tvu : v;
                        ix = sw ? tiu : ix;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(accfree));
            // merge the column groups of each row (scratch in the activation
            // buffer: the last layer's products have read it)
            constexpr int SW = 2 * TM + 2;
            if (C::CG > 1) {
                float *my = scratch + (size_t)j * SW * MT + rit;
#pragma unroll
                for (int q = 0; q < TM; ++q) {
                    my[q * MT] = tv[q];
                    my[(TM + q) * MT] = __int_as_float(ti[q]);
                }
                my[2 * TM * MT] = mx;
                my[(2 * TM + 1) * MT] = se;
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(mready));
            }
            if (j == 0) {
                if (C::CG > 1 && !__all_sync(0xffffffffu, mbar_wait(smem_u32(mready), it & 1, abort_flag))) break;
                for (int jj = 1; jj < C::CG; ++jj) {
                    const float *o = scratch + (size_t)jj * SW * MT + rit;
                    const float omx = o[2 * TM * MT], ose = o[(2 * TM + 1) * MT];
                    const float M = fmaxf(mx, omx);
                    se = se * __expf(mx - M) + ose * __expf(omx - M);
                    mx = M;
#pragma unroll
                    for (int q = 0; q < TM; ++q) topm_insert<TM>(tv, ti, o[q * MT], __float_as_int(o[(TM + q) * MT]));
                }
                if (row < n) {
                    float mass = 0.0f;
#pragma unroll
                    for (int q = 0; q < TM; ++q)
                        if (q < topm) {
                            mass += __expf(tv[q] - mx);
                            cand[(size_t)row * topm + q] = ti[q];
                        }
                    pmass[row] = mass / se;
                }
                if (C::CG > 1) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(mdone));
                }
            }
            // the next tile's activations overwrite the scratch
            if (C::CG > 1 && !__all_sync(0xffffffffu, mbar_wait(smem_u32(mdone), it & 1, abort_flag))) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(err, 1);
}

// ============================================================================
// Scores of (patch, candidate) pairs on the tensor cores, grouped by
// component: a CTA takes one work item (up to 128 pairs proposing component
// k), gathers their DC-free patches from the image into shared memory as
// split BF16 operands (hi + lo, written in the 128-byte-swizzled K-major
// layout), loads the component's split scaled basis Ubar_k sqrt|q_k| (64 rows,
// hi + lo) by TMA, and accumulates hi*hi + lo*hi + hi*lo (the split form of
// the exhaustive pass, with the same error bound) into 64 TMEM columns.  Each
// epilogue thread finishes its pair's score of Eq. 14:
//   cst_k + t_k |z|^2 + sgn_k sum_{j < r_k} c_j^2.
// ============================================================================
constexpr int PS_T = 128;
constexpr int PS_TILE = PS_T * 128;   // 16 KB: [128 rows][64] BF16
constexpr int PS_B = 64 * 128;        // 8 KB: [64 rows][64] BF16
constexpr int PS_SMEM = 1024 + 2 * PS_TILE + 2 * PS_B + 32 + 3 * PS_T * 4;

__global__ void __launch_bounds__(PS_T)
k_pair_score_tc(const __grid_constant__ CUtensorMap mapBs, const __grid_constant__ CUtensorMap mapBlo,
                const float *__restrict__ xhat, int H, int W, const int *__restrict__ anchors,
                const int *__restrict__ perm, const int4 *__restrict__ items, int topm,
                const int *__restrict__ rowlist, const int *__restrict__ roff, const int *__restrict__ rk_,
                Tables tab, const float *__restrict__ zz, float *__restrict__ pscore, int *__restrict__ err)
{
    pdl_enter();
    const int nitems = items[0].w;
    if ((int)blockIdx.x >= nitems) return;
    extern __shared__ __align__(1024) unsigned char ps_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)ps_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *Ahi = smem, *Alo = smem + PS_TILE, *Bhi = smem + 2 * PS_TILE, *Blo = Bhi + PS_B;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(Blo + PS_B);  // [0] B loaded, [1] MMA done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    int *s_anchor = reinterpret_cast<int *>(tslot + 2), *s_pair = s_anchor + PS_T, *s_row = s_pair + PS_T;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const int pr_ = lane >> 2, pc_ = 2 * (lane & 3);
    // work items b, b + gridDim.x, ...; the barriers' phase is the local iteration's parity
    for (int item = blockIdx.x, iter = 0; item < nitems; item += gridDim.x, ++iter) {
        const int4 it = items[1 + item];
        const int k = it.x, first = it.y, cnt_p = it.z;
        const uint32_t ph = (uint32_t)(iter & 1);
        if (threadIdx.x == 0) {
            const uint32_t b = smem_u32(&bars[0]);
            mbar_expect_tx(b, 2 * PS_B);
            tma_load_2d(smem_u32(Bhi), &mapBs, 0, roff[k], b);
            tma_load_2d(smem_u32(Blo), &mapBlo, 0, roff[k], b);
        }
        // gather: every thread first resolves one row's pair -> patch -> anchor;
        // then warp w fills rows 32w .. 32w+31, eight rows' loads in flight at a
        // time, lane l holding patch elements 2l and 2l + 1 (patch row l / 4)
        if (threadIdx.x < cnt_p) {
            const int pr = perm[first + threadIdx.x];
            const int i = rowlist ? rowlist[pr / topm] : pr / topm;
            s_pair[threadIdx.x] = pr;
            s_row[threadIdx.x] = i;
            s_anchor[threadIdx.x] = anchors ? anchors[i] : i;
        }
        __syncthreads();
        for (int rr = 0; rr < 32; rr += 8) {
            float xa[8], xb[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = 32 * warp + rr + u;
                xa[u] = xb[u] = 0.0f;
                if (t < cnt_p) {
                    const int a = s_anchor[t];
                    const int ai = a / W, aj = a % W;
                    int r = ai + pr_, c0 = aj + pc_, c1 = c0 + 1;
                    if (r >= H) r -= H;
                    if (c0 >= W) c0 -= W;
                    if (c1 >= W) c1 -= W;
                    xa[u] = xhat[(size_t)r * W + c0];
                    xb[u] = xhat[(size_t)r * W + c1];
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = 32 * warp + rr + u;
                float sum = xa[u] + xb[u];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                const float mu = t < cnt_p ? sum * (1.0f / PD) : 0.0f;
                const float z0 = xa[u] - mu, z1 = xb[u] - mu;
                const __nv_bfloat162 h = __floats2bfloat162_rn(z0, z1);
                const __nv_bfloat162 l = __floats2bfloat162_rn(z0 - __low2float(h), z1 - __high2float(h));
                // elements 2l, 2l+1: bytes 4l..4l+3 of the row, 16-byte chunk l / 4 swizzled by t mod 8
                const uint32_t o = t * 128 + ((((uint32_t)lane >> 2) ^ (t & 7)) << 4) + 4 * (lane & 3);
                *reinterpret_cast<__nv_bfloat162 *>(Ahi + o) = h;
                *reinterpret_cast<__nv_bfloat162 *>(Alo + o) = l;
            }
        }
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            if (mbar_wait(smem_u32(&bars[0]), ph, abort_flag)) {
                tc_fence_after();
                const uint32_t idesc = idesc_f16(PS_T, 64, 1);
                const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t o = 32 * kk;
                    mma_f16(tbase, sdesc_sw128(ah + o), sdesc_sw128(bh + o), idesc, kk ? 1u : 0u);
                    mma_f16(tbase, sdesc_sw128(al + o), sdesc_sw128(bh + o), idesc, 1u);
                    mma_f16(tbase, sdesc_sw128(ah + o), sdesc_sw128(bl + o), idesc, 1u);
                }
                mma_commit(smem_u32(&bars[1]));
            }
        }
        __syncwarp();
        const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&bars[1]), ph, abort_flag));
        tc_fence_after();
        if (ok) {
            uint32_t r[64];
            tmem_ld_all<64>(tbase + ((uint32_t)(32 * warp) << 16), r);
            const int t = 32 * warp + lane, rk = rk_[k];
            float sq = 0.0f;
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                const float c = __uint_as_float(r[j]);
                if (j < rk) sq = fmaf(c, c, sq);
            }
            if (t < cnt_p) pscore[s_pair[t]] = tab.cst_hi[k] + tab.t_hi[k] * zz[s_row[t]] + tab.sgn[k] * sq;
        }
        tc_fence_before();
        // the next item overwrites the operands and the accumulator
        if (__syncthreads_or(!ok)) break;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tbase) : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(err, 1);
}

// Per entry: best and second-best rescored candidate (lowest index on ties);
// undecided patches (proposal mass below pmin, or a top-2 gap within the
// split-BF16 error bound, or an absent first candidate) are listed for the
// next pass.  Entry f is patch f, or patch list[f] of a device list (count
// *nlist); a negative candidate is absent; pmass and nfallback are nullable.
__global__ void k_prop_combine(int n, const int *__restrict__ list, const int *__restrict__ nlist, int topm,
                               const int *__restrict__ cand, const float *__restrict__ pscore,
                               const float *__restrict__ pmass, float pmin, const float *__restrict__ zz,
                               const float *__restrict__ tmax, float tau_abs, float tau_rel,
                               int *__restrict__ kstar, float *__restrict__ gap, int *__restrict__ flag,
                               int *__restrict__ nflag, long long *__restrict__ nfallback)
{
    pdl_enter();
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = list ? min(n, *nlist) : n;
    bool unsure = false;
    if (f < total) {
        const int i = list ? list[f] : f;
        float s1 = FLT_MAX, s2 = FLT_MAX;
        int k1 = 0x7fffffff;
        for (int q = 0; q < topm; ++q) {
            const int k = cand[(size_t)f * topm + q];
            if (k < 0) continue;
            const float s = pscore ? pscore[(size_t)f * topm + q] : 0.0f;
            if (s < s1 || (s == s1 && k < k1)) {
                s2 = s1;
                s1 = s;
                k1 = k;
            } else if (s < s2) {
                s2 = s;
            }
        }
        const float gp = s2 - s1;
        if (k1 != 0x7fffffff) {
            kstar[i] = k1;
            gap[i] = gp;
        }
        unsure = k1 == 0x7fffffff || (pmass && !(pmass[i] >= pmin)) ||
                 !(gp >= tau_abs + tau_rel * zz[i] * tmax[0]);
        if (unsure) flag[atomicAdd(nflag, 1)] = i;
    }
    const unsigned b = __ballot_sync(0xffffffffu, unsure);
    if (nfallback && (threadIdx.x & 31) == 0 && b)
        atomicAdd((unsigned long long *)nfallback, (unsigned long long)__popc(b));
}

epll_status ensure_prop_ws(epll_gmm *g, int n)
{
    Workspace &ws = g->ws;
    const size_t N = ws.capN;
    if (ws.cand && ws.prop_cap >= N) return EPLL_OK;
    void *ptrs[] = {ws.cand, ws.pmass, ws.pperm, ws.pitems, ws.pscore};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    cudaError_t e = cudaSuccess;
    auto A = [&](void **q, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(q, bytes); };
    A((void **)&ws.cand, N * TOPM_MAX * 4); A((void **)&ws.pmass, N * 4); A((void **)&ws.pperm, N * TOPM_MAX * 4);
    A((void **)&ws.pitems, (2 + N * TOPM_MAX / 128 + (size_t)g->K) * sizeof(int4));
    A((void **)&ws.pscore, N * TOPM_MAX * 4);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(EPLL_ENOMEM, std::string("proposal workspace: ") + cudaGetErrorString(e));
    }
    ws.prop_cap = N;
    (void)n;
    return EPLL_OK;
}

constexpr int FM_EW = 16;  // epilogue warps of the fused kernel

epll_status launch_proposal_topm(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                                 const float *ibeta, cudaStream_t st)
{
    const epll_proposal *p = g->prop;
    Workspace &ws = g->ws;
    epll_status s;
    if ((s = ensure_prop_ws(g, n))) return s;
    const int rows = (n + MT - 1) / MT * MT;
    // DC-free patches as split BF16 operands (the network reads the hi part;
    // the estimation reuses both), |z|^2 and the means
    if ((s = launch_extract_split(g, xhat, H, W, anchors, n, st))) return s;
    const int n3 = (p->K + 15) / 16 * 16;
    CUtensorMap mz, w1, w2, w3;
    if ((s = make_map(&mz, ws.Zb, rows, MT))) return s;
    if ((s = make_map(&w1, p->W1b, HID, HID))) return s;
    if ((s = make_map_wide(&w2, p->W2b, HID, HID, HID))) return s;
    if ((s = make_map_wide(&w3, p->W3b, HID, n3, HID))) return s;
    using Cf = FmCfg<FM_EW>;
    const int topm = g->prop_topm;
    auto kern = topm == 1 ? k_mlp_fused<FM_EW, 1>
                          : (topm == 2 ? k_mlp_fused<FM_EW, 2> : (topm <= 4 ? k_mlp_fused<FM_EW, 4> : k_mlp_fused<FM_EW, 8>));
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        EPLL_CU(cudaGetDevice(&dev));
        EPLL_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        EPLL_CU(cudaFuncSetAttribute(k_mlp_fused<FM_EW, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM));
        EPLL_CU(cudaFuncSetAttribute(k_mlp_fused<FM_EW, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM));
        EPLL_CU(cudaFuncSetAttribute(k_mlp_fused<FM_EW, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM));
        EPLL_CU(cudaFuncSetAttribute(k_mlp_fused<FM_EW, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM));
    }
    const int ntiles = rows / MT;
    const int grid = ntiles < sms ? ntiles : sms;
    prof_begin(g, st);
    kern<<<grid, Cf::THREADS, Cf::SMEM, st>>>(mz, w1, w2, w3, n, p->K, n3, p->wr, ibeta, topm, ws.cand, ws.pmass,
                                              cnt(g, CNT_ERR));
    prof_end(g, st, n, 2.0 * ((double)HID * PD + (double)HID * HID + (double)HID * p->K));
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

epll_status launch_pair_scores(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n, int m,
                               const int *list, const int *nlist, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int npairs = n * m;
    epll_status s;
    if ((s = group_by_component(g, ws.cand, npairs, ws.pperm, ws.pitems, st, list ? nlist : nullptr, m))) return s;
    static bool attr = false;
    if (!attr) {
        EPLL_CU(cudaFuncSetAttribute(k_pair_score_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, PS_SMEM));
        attr = true;
    }
    CUtensorMap bs, bslo;
    if ((s = make_map(&bs, g->tab.Bs, g->Rtot, 64))) return s;
    if ((s = make_map(&bslo, g->tab.Bs_lo, g->Rtot, 64))) return s;
    // persistent over the work items (their count is known on the device only)
    const int max_items = (npairs + PS_T - 1) / PS_T + g->K;
    const int grid = max_items < 152 * 4 ? max_items : 152 * 4;
    EPLL_CU(launch_pdl(k_pair_score_tc, dim3(grid), dim3(PS_T), PS_SMEM, st, bs, bslo, xhat, H, W, anchors, ws.pperm, ws.pitems, m, list,
                                                 g->d_roff, g->d_r, g->tab, ws.zz, ws.pscore, cnt(g, CNT_ERR)));
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

epll_status launch_cand_combine(epll_gmm *g, int n, int m, const int *list, const int *nlist, float tau_abs,
                                int *flag, int *nflag, cudaStream_t st)
{
    Workspace &ws = g->ws;
    EPLL_CU(launch_pdl(k_prop_combine, dim3((n + 255) / 256), dim3(256), 0, st, n, list, nlist, m, ws.cand, ws.pscore, nullptr, 0.0f, ws.zz,
                                                   g->tab.tmax, tau_abs, SPLIT_REL, ws.kstar, ws.gap, flag, nflag,
                                                   nullptr));
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

epll_status launch_select_proposal(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                                   float tau_abs, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int topm = g->prop_topm;
    epll_status s;
    if ((s = launch_proposal_topm(g, xhat, H, W, anchors, n, g->tab.ibeta, st))) return s;
    // exact FP32 scores of the proposed (patch, component) pairs; a single
    // proposal is the selection (its gap is reported as FLT_MAX)
    if (topm > 1 && (s = launch_pair_scores(g, xhat, H, W, anchors, n, topm, nullptr, nullptr, st))) return s;
    int *nflag1 = cnt(g, CNT_NFLAG1);
    EPLL_CU(cudaMemsetAsync(nflag1, 0, sizeof(int), st));
    EPLL_CU(launch_pdl(k_prop_combine, dim3((n + 255) / 256), dim3(256), 0, st, n, nullptr, nullptr, topm, ws.cand, topm > 1 ? ws.pscore : nullptr, ws.pmass,
                                                   g->prop_pmin, ws.zz,
                                                   g->tab.tmax, tau_abs, SPLIT_REL, ws.kstar, ws.gap, ws.flag1,
                                                   nflag1, ws.ctr + 1));
    EPLL_LAUNCHED(g);
    // exhaustive split-BF16 pass over the undecided patches
    return launch_split_pass(g, xhat, H, W, anchors, n, ws.flag1, nflag1, tau_abs, st);
}

}  // namespace epll

using namespace epll;

extern "C" {

size_t epll_proposal_size(int K) { return K >= 1 ? prop_size(K) : 0; }

void epll_proposal_free(epll_proposal *p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    void *ptrs[] = {p->theta, p->mom1, p->mom2, p->grad, p->wr, p->W1b, p->W2b, p->W3b, p->X, p->cond,
                    p->A1, p->H1, p->A2, p->H2, p->L, p->dH, p->dA, p->loss, p->partial};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete p;
}

epll_status epll_proposal_create(int K, uint64_t seed, epll_proposal **out)
{
    if (!out) return fail(EPLL_EINVAL, "null output pointer");
    *out = nullptr;
    if (K < 2 || K > HID) return fail(EPLL_EINVAL, "proposal networks serve 2..256 components");
    epll_proposal *p = new epll_proposal();
    p->K = K;
    p->np = prop_size(K);
    cudaError_t e = cudaSuccess;
    auto A = [&](void **q, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(q, bytes); };
    A((void **)&p->theta, p->np * 4); A((void **)&p->mom1, p->np * 4); A((void **)&p->mom2, p->np * 4);
    A((void **)&p->grad, p->np * 4); A((void **)&p->wr, p->np * 4);
    A((void **)&p->W1b, HID * PD * 2); A((void **)&p->W2b, HID * HID * 2); A((void **)&p->W3b, HID * HID * 2);
    A((void **)&p->loss, 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        epll_proposal_free(p);
        return fail(EPLL_ENOMEM, "proposal allocation failed");
    }
    // He-style initialisation from counter-based draws (splitmix64 + Box-Muller)
    std::vector<float> th(p->np, 0.0f);
    auto mix = [](uint64_t z) {
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        return z ^ (z >> 31);
    };
    auto normal = [&](uint64_t i) {
        const double u1 = ((mix(seed + 2 * i + 1) >> 11) + 0.5) * 0x1.0p-53;
        const double u2 = ((mix(seed + 2 * i + 2) >> 11) + 0.5) * 0x1.0p-53;
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (size_t i = OFF_W1; i < OFF_B1; ++i) th[i] = (float)(normal(i) * std::sqrt(2.0 / PD));
    for (size_t i = OFF_W2; i < OFF_B2; ++i) th[i] = (float)(normal(i) * std::sqrt(2.0 / HID));
    for (size_t i = OFF_W3; i < off_b3(K); ++i) th[i] = (float)(normal(i) * std::sqrt(1.0 / HID));
    auto C = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    C(cudaMemcpy(p->theta, th.data(), p->np * 4, cudaMemcpyHostToDevice));
    C(cudaMemset(p->mom1, 0, p->np * 4)); C(cudaMemset(p->mom2, 0, p->np * 4));
    C(cudaMemset(p->W3b, 0, HID * HID * 2));
    if (e != cudaSuccess || refresh(p, 0) != EPLL_OK || cudaDeviceSynchronize() != cudaSuccess) {
        epll_proposal_free(p);
        return fail(EPLL_ECUDA, "proposal initialisation failed");
    }
    *out = p;
    return EPLL_OK;
}

epll_status epll_proposal_get(const epll_proposal *p, float *params)
{
    if (!p || !params) return fail(EPLL_EINVAL, "null argument");
    EPLL_CU(cudaMemcpy(params, p->theta, p->np * 4, cudaMemcpyDeviceToHost));
    return EPLL_OK;
}

epll_status epll_proposal_set(epll_proposal *p, const float *params)
{
    if (!p || !params) return fail(EPLL_EINVAL, "null argument");
    for (size_t i = 0; i < p->np; ++i)
        if (!std::isfinite(params[i])) return fail(EPLL_EINVAL, "parameters must be finite");
    EPLL_CU(cudaMemcpy(p->theta, params, p->np * 4, cudaMemcpyHostToDevice));
    EPLL_CU(cudaMemset(p->mom1, 0, p->np * 4));
    EPLL_CU(cudaMemset(p->mom2, 0, p->np * 4));
    p->step = 0;
    epll_status s = refresh(p, 0);
    if (s) return s;
    EPLL_CU(cudaDeviceSynchronize());
    return EPLL_OK;
}

static epll_status check_batch(const epll_proposal *p, const Batch &d)
{
    if (!p || !d.images || !d.img_idx || !d.anchors || !d.log_ib || !d.labels)
        return fail(EPLL_EINVAL, "null argument");
    if (d.n_img < 1 || d.H < PS || d.W < PS || (long long)d.H * d.W > (1LL << 26))
        return fail(EPLL_EINVAL, "images must be n_img >= 1 of 8 x 8 .. 2^26 pixels");
    if (d.B < 1 || d.B > (1 << 20)) return fail(EPLL_EINVAL, "batch size must be in 1..2^20");
    if (d.n_all < d.B || (!d.sel && d.n_all != d.B)) return fail(EPLL_EINVAL, "n_all must be >= B (== B without sel)");
    return EPLL_OK;
}

// Reads the loss and the invalid-sample flag (synchronises st).
static epll_status read_loss(epll_proposal *p, float *loss, cudaStream_t st)
{
    float h[3];
    EPLL_CU(cudaMemcpyAsync(h, p->loss, sizeof(h), cudaMemcpyDeviceToHost, st));
    EPLL_CU(cudaStreamSynchronize(st));
    int bad, tc_err;
    std::memcpy(&bad, &h[1], sizeof(int));
    std::memcpy(&tc_err, &h[2], sizeof(int));
    if (tc_err) return fail(EPLL_ETIMEOUT, "a training GEMM gave up on a bounded wait");
    if (bad) return fail(EPLL_EINVAL, "a sample had an out-of-range image index, anchor, label or log(1/beta)");
    *loss = h[0];
    return EPLL_OK;
}

epll_status epll_proposal_grad(epll_proposal *p, const float *images, int n_img, int H, int W, const int *img_idx,
                               const int *anchors, const float *log_ib, const int *labels, const int *sel,
                               int n_all, int B, float *grad, float *loss, void *stream)
{
    const Batch d{images, n_img, H, W, img_idx, anchors, log_ib, labels, sel, n_all, B};
    epll_status s;
    if ((s = check_batch(p, d))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = forward_backward(p, d, st))) return s;
    if (grad) EPLL_CU(cudaMemcpyAsync(grad, p->grad, p->np * 4, cudaMemcpyDeviceToDevice, st));
    return loss ? read_loss(p, loss, st) : EPLL_OK;
}

epll_status epll_proposal_train(epll_proposal *p, const float *images, int n_img, int H, int W,
                                const int *img_idx, const int *anchors, const float *log_ib, const int *labels,
                                const int *sel, int n_all, int B, float lr, float weight_decay, float *loss,
                                void *stream)
{
    const Batch d{images, n_img, H, W, img_idx, anchors, log_ib, labels, sel, n_all, B};
    epll_status s;
    if ((s = check_batch(p, d))) return s;
    if (!(lr > 0.0f) || !std::isfinite(lr) || !(weight_decay >= 0.0f) || !std::isfinite(weight_decay))
        return fail(EPLL_EINVAL, "bad learning rate or weight decay");
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = forward_backward(p, d, st))) return s;
    ++p->step;
    const float c1 = 1.0f - (float)std::pow(0.9, (double)p->step), c2 = 1.0f - (float)std::pow(0.999, (double)p->step);
    k_adamw<<<(int)((p->np + 255) / 256), 256, 0, st>>>(p->theta, p->grad, p->mom1, p->mom2, (long)p->np, p->K, lr,
                                                         weight_decay, c1, c2);
    EPLL_CU(cudaGetLastError());
    if ((s = refresh(p, st))) return s;
    return loss ? read_loss(p, loss, st) : EPLL_OK;
}

__global__ void k_set_f32(float *p, float v) { *p = v; }

epll_status epll_proposal_topm(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                               double beta, int *cand, float *pmass, void *stream)
{
    if (!g) return fail(EPLL_EINVAL, "null model handle");
    if (!g->prop) return fail(EPLL_EINVAL, "no proposal network attached");
    if (!xhat || !cand) return fail(EPLL_EINVAL, "null pointer");
    if (H < PS || W < PS || (long long)H * W > (1LL << 26)) return fail(EPLL_EINVAL, "bad image size");
    if (!anchors) n = H * W;
    if (n < 1 || (long long)n > (long long)H * W) return fail(EPLL_EINVAL, "n must be in 1..H*W");
    if (!(beta > 0.0) || !std::isfinite(beta)) return fail(EPLL_EINVAL, "beta must be positive");
    epll_status s;
    if ((s = ensure_workspace(g, (size_t)H * W))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace &ws = g->ws;
    EPLL_CU(cudaMemsetAsync(cnt(g, CNT_ERR), 0, sizeof(int), st));
    float *ib = ws.red;  // scratch scalar
    k_set_f32<<<1, 1, 0, st>>>(ib, (float)(1.0 / beta));
    EPLL_LAUNCHED(g);
    if ((s = launch_proposal_topm(g, xhat, H, W, anchors, n, ib, st))) return s;
    const int topm = g->prop_topm;
    EPLL_CU(cudaMemcpyAsync(cand, ws.cand, sizeof(int) * (size_t)n * topm, cudaMemcpyDeviceToDevice, st));
    if (pmass) EPLL_CU(cudaMemcpyAsync(pmass, ws.pmass, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    return EPLL_OK;
}

epll_status epll_gmm_attach_proposal(epll_gmm *g, const epll_proposal *p, int topm, float pmin)
{
    if (!g) return fail(EPLL_EINVAL, "null model handle");
    if (p && p->K != g->K) return fail(EPLL_EINVAL, "proposal and model have different K");
    if (p && (topm < 1 || topm > TOPM_MAX || topm > p->K)) return fail(EPLL_EINVAL, "topm must be in 1..min(8, K)");
    if (!(pmin >= 0.0f && pmin <= 1.0f)) return fail(EPLL_EINVAL, "pmin must be in [0, 1]");
    g->prop = p;
    g->prop_topm = topm;
    g->prop_pmin = pmin;
    return EPLL_OK;
}

}  // extern "C"
