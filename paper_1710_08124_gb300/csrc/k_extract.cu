// Extraction of the sampled patches as tensor-core operands (Algorithm 1,
// first step): DC-free patches as 16-bit operands (hi, and lo for the split
// variant) or 8-bit E4M3 rows with a per-row scale, their FP32 squared norms
// and (optionally) their means.  Rows up to the next multiple of 128 are
// zero-filled so the last tile's rows are defined.
#include "epll_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

namespace epll {

__device__ __forceinline__ uint8_t to_e4m3(float v)
{
    return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}
// Row i of the operand is sampled patch i, or patch rowmap[i] when a row map
// (a device list with device count *n_dev) is given.  mu_out (nullable)
// receives each row's patch mean; Zf (nullable) an FP16 copy of the rows
// (written beside BF16 split rows for an FP16 first pass).
// fmt 3: 8-bit E4M3 operands scaled per row (max |z| -> 448), the square of
// the scale in zsc2; Zhi is then read as bytes.
//
// Eight threads per patch, one per patch row: a thread loads its row's eight
// pixels (three aligned 16-byte loads away from the right edge), the patch
// sums (mean, |z|^2, max |z|) are reduced over the eight lanes of the patch,
// and each thread writes its row's eight operands as one 16-byte store
// (8 bytes for E4M3), so the eight lanes of a patch write its 128-byte
// operand row contiguously.
constexpr int EX_THREADS = 256;
constexpr int EX_PATCHES = EX_THREADS / PS;  // patches per block and pass

__device__ __forceinline__ float sum8(float v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    return v;
}
__device__ __forceinline__ float max8(float v)
{
    v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 1));
    v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 2));
    v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 4));
    return v;
}
// two values rounded to nearest (even) as one packed 16-bit pair (one
// conversion instruction; the same roundings as two scalar conversions)
__device__ __forceinline__ uint32_t pack16(float a, float b, int fmt)
{
    if (fmt == 2) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ float lo16f(uint32_t p, int fmt)
{
    return fmt == 2 ? __half2float(__ushort_as_half((unsigned short)(p & 0xffffu))) : __uint_as_float(p << 16);
}
__device__ __forceinline__ float hi16f(uint32_t p, int fmt)
{
    return fmt == 2 ? __half2float(__ushort_as_half((unsigned short)(p >> 16))) : __uint_as_float(p & 0xffff0000u);
}
__device__ __forceinline__ uint4 pack16x8(const float *v, int fmt)
{
    return make_uint4(pack16(v[0], v[1], fmt), pack16(v[2], v[3], fmt), pack16(v[4], v[5], fmt),
                      pack16(v[6], v[7], fmt));
}

__global__ void __launch_bounds__(EX_THREADS)
k_extract_tc(const float *__restrict__ xhat, int H, int W, const int *__restrict__ anchors, int n,
             const int *__restrict__ rowmap, const int *__restrict__ n_dev, int fmt, int split,
             uint16_t *__restrict__ Zhi, uint16_t *__restrict__ Zlo, float *__restrict__ zz,
             float *__restrict__ zsc2, float *__restrict__ mu_out, uint16_t *__restrict__ Zf)
{
    pdl_enter();
    const int u = threadIdx.x & (PS - 1);  // patch row of this thread
    // image rows start on 16-byte boundaries (vector loads allowed)
    const bool aligned = (W & 3) == 0 && ((uintptr_t)xhat & 15) == 0;
    if (n_dev) n = *n_dev;
    const int rows = (n + 127) / 128 * 128;
    // grid-stride over blocks of EX_PATCHES rows (a listed subset launches a capped grid)
    for (int i = blockIdx.x * EX_PATCHES + (threadIdx.x >> 3); i - (int)(threadIdx.x >> 3) < rows;
         i += gridDim.x * EX_PATCHES) {
        float x[PS];
        const bool live = i < n;
        if (live) {
            const int p = rowmap ? rowmap[i] : i;
            const int a = anchors ? anchors[p] : p;
            const int ai = a / W, aj = a - ai * W;
            int r = ai + u;
            if (r >= H) r -= H;
            const float *src = xhat + (size_t)r * W;
            const int base = aj & ~3, sh = aj & 3;
            if (aligned && base + 12 <= W) {
                // three aligned 16-byte loads cover the row's eight pixels
                const float4 *s4 = reinterpret_cast<const float4 *>(src + base);
                const float4 f0 = s4[0], f1 = s4[1];
                const float4 f2 = sh ? s4[2] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                const float F[12] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w, f2.x, f2.y, f2.z, f2.w};
#pragma unroll
                for (int v = 0; v < PS; ++v)
                    x[v] = sh == 0 ? F[v] : sh == 1 ? F[v + 1] : sh == 2 ? F[v + 2] : F[v + 3];
            } else {
#pragma unroll
                for (int v = 0; v < PS; ++v) {
                    int c = aj + v;
                    if (c >= W) c -= W;
                    x[v] = src[c];
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < PS; ++v) x[v] = 0.0f;
        }
        float s = 0.0f;
#pragma unroll
        for (int v = 0; v < PS; ++v) s += x[v];
        const float mu = sum8(s) * (1.0f / PD);
        float z[PS], q = 0.0f;
#pragma unroll
        for (int v = 0; v < PS; ++v) {
            z[v] = live ? x[v] - mu : 0.0f;
            q = fmaf(z[v], z[v], q);
        }
        q = sum8(q);
        if (i >= rows) continue;  // after the shuffles: every lane of the warp took part
        const size_t off = (size_t)i * PD + (size_t)u * PS;
        if (fmt == 3) {
            float m = 0.0f;
#pragma unroll
            for (int v = 0; v < PS; ++v) m = fmaxf(m, fabsf(z[v]));
            m = max8(m);
            const float sc = m > 0.0f ? m / 448.0f : 1.0f;
            uint32_t b[2] = {0u, 0u};
#pragma unroll
            for (int v = 0; v < PS; ++v) b[v >> 2] |= (uint32_t)to_e4m3(z[v] / sc) << (8 * (v & 3));
            *reinterpret_cast<uint2 *>(reinterpret_cast<uint8_t *>(Zhi) + off) = make_uint2(b[0], b[1]);
            if (u == 0 && live) {
                zz[i] = q;
                zsc2[i] = sc * sc;
            }
        } else {
            const uint4 hi = pack16x8(z, fmt);
            *reinterpret_cast<uint4 *>(Zhi + off) = hi;
            if (split) {
                const uint32_t hw[4] = {hi.x, hi.y, hi.z, hi.w};
                float lo[PS];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    lo[2 * q] = z[2 * q] - lo16f(hw[q], fmt);
                    lo[2 * q + 1] = z[2 * q + 1] - hi16f(hw[q], fmt);
                }
                *reinterpret_cast<uint4 *>(Zlo + off) = pack16x8(lo, fmt);
            }
            if (Zf) *reinterpret_cast<uint4 *>(Zf + off) = pack16x8(z, 2);
            if (u == 0 && live) {
                zz[i] = q;
                if (mu_out) mu_out[i] = mu;
            }
        }
    }
}

// Blocks for `rows` operand rows (a listed subset: capped, the kernel strides).
static inline int ex_grid(int rows, bool listed)
{
    const int b = (rows + EX_PATCHES - 1) / EX_PATCHES;
    return listed && b > 152 * 2 ? 152 * 2 : b;
}

epll_status launch_extract(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                           const int *rowmap, const int *n_dev, int fmt, int split, uint16_t *Zhi, uint16_t *Zlo,
                           float *zz, float *zsc2, float *mu, cudaStream_t st, uint16_t *Zf)
{
    const int rows = (n + 127) / 128 * 128;
    EPLL_CU(launch_pdl(k_extract_tc, dim3(ex_grid(rows, n_dev != nullptr)), dim3(EX_THREADS), 0, st, xhat, H, W,
                       anchors, n, rowmap, n_dev, fmt, split, Zhi, Zlo, zz, zsc2, mu, Zf));
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

epll_status launch_extract_split(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                                 cudaStream_t st)
{
    Workspace &ws = g->ws;
    return launch_extract(g, xhat, H, W, anchors, n, nullptr, nullptr, 1, 1, ws.Zb, ws.Zb + ws.zrows * PD, ws.zz,
                          nullptr, ws.mu, st);
}

}  // namespace epll
