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

__device__ __forceinline__ float warp_sum_tc(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max_tc(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ uint8_t to_e4m3(float v)
{
    return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ uint16_t to16(float v, int fmt)
{
    return fmt == 2 ? __half_as_ushort(__float2half_rn(v)) : __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float from16(uint16_t v, int fmt)
{
    return fmt == 2 ? __half2float(__ushort_as_half(v)) : __bfloat162float(__ushort_as_bfloat16(v));
}

// Row i of the operand is sampled patch i, or patch rowmap[i] when a row map
// (a device list with device count *n_dev) is given.  mu_out (nullable)
// receives each row's patch mean; Zf (nullable) an FP16 copy of the rows
// (written beside BF16 split rows for an FP16 first pass).
// fmt 3: 8-bit E4M3 operands scaled per row (max |z| -> 448), the square of
// the scale in zsc2; Zhi is then read as bytes.
constexpr int EX_ROWS = 4;  // rows per warp and pass: their loads are issued together
__global__ void __launch_bounds__(128)
k_extract_tc(const float *__restrict__ xhat, int H, int W, const int *__restrict__ anchors, int n,
             const int *__restrict__ rowmap, const int *__restrict__ n_dev, int fmt, int split,
             uint16_t *__restrict__ Zhi, uint16_t *__restrict__ Zlo, float *__restrict__ zz,
             float *__restrict__ zsc2, float *__restrict__ mu_out, uint16_t *__restrict__ Zf)
{
    const int lane = threadIdx.x & 31;
    if (n_dev) n = *n_dev;
    const int rows = (n + 127) / 128 * 128;
    // grid-stride over groups of EX_ROWS rows (a listed subset launches a capped grid)
    for (int base = (blockIdx.x * 4 + (threadIdx.x >> 5)) * EX_ROWS; base < rows;
         base += gridDim.x * 4 * EX_ROWS) {
        float x0[EX_ROWS], x1[EX_ROWS];
#pragma unroll
        for (int u = 0; u < EX_ROWS; ++u) {
            const int i = base + u;
            x0[u] = x1[u] = 0.0f;
            if (i < n) {
                const int p = rowmap ? rowmap[i] : i;
                const int a = anchors ? anchors[p] : p;
                const int ai = a / W, aj = a % W;
                int r0 = ai + (lane >> 3), r1 = r0 + 4, c = aj + (lane & 7);
                if (r0 >= H) r0 -= H;
                if (r1 >= H) r1 -= H;
                if (c >= W) c -= W;
                x0[u] = xhat[(size_t)r0 * W + c];
                x1[u] = xhat[(size_t)r1 * W + c];
            }
        }
#pragma unroll
        for (int u = 0; u < EX_ROWS; ++u) {
            const int i = base + u;
            float z0 = 0.0f, z1 = 0.0f, q = 0.0f, mu = 0.0f;
            if (i < n) {
                mu = warp_sum_tc(x0[u] + x1[u]) * (1.0f / PD);
                z0 = x0[u] - mu;
                z1 = x1[u] - mu;
                q = warp_sum_tc(z0 * z0 + z1 * z1);
            }
            if (fmt == 3) {
                const float m = warp_max_tc(fmaxf(fabsf(z0), fabsf(z1)));
                const float sc = m > 0.0f ? m / 448.0f : 1.0f;
                uint8_t *Z8 = reinterpret_cast<uint8_t *>(Zhi);
                Z8[(size_t)i * PD + lane] = to_e4m3(z0 / sc);
                Z8[(size_t)i * PD + lane + 32] = to_e4m3(z1 / sc);
                if (lane == 0 && i < n) {
                    zz[i] = q;
                    zsc2[i] = sc * sc;
                }
            } else {
                const uint16_t h0 = to16(z0, fmt), h1 = to16(z1, fmt);
                Zhi[(size_t)i * PD + lane] = h0;
                Zhi[(size_t)i * PD + lane + 32] = h1;
                if (split) {
                    Zlo[(size_t)i * PD + lane] = to16(z0 - from16(h0, fmt), fmt);
                    Zlo[(size_t)i * PD + lane + 32] = to16(z1 - from16(h1, fmt), fmt);
                }
                if (Zf) {
                    Zf[(size_t)i * PD + lane] = to16(z0, 2);
                    Zf[(size_t)i * PD + lane + 32] = to16(z1, 2);
                }
                if (lane == 0 && i < n) {
                    zz[i] = q;
                    if (mu_out) mu_out[i] = mu;
                }
            }
        }
    }
}

// Blocks for `rows` operand rows (a listed subset: capped, the kernel strides).
static inline int ex_grid(int rows, bool listed)
{
    const int b = (rows + 4 * EX_ROWS - 1) / (4 * EX_ROWS);
    return listed && b > 152 * 16 ? 152 * 16 : b;
}

epll_status launch_extract(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                           const int *rowmap, const int *n_dev, int fmt, int split, uint16_t *Zhi, uint16_t *Zlo,
                           float *zz, float *zsc2, float *mu, cudaStream_t st, uint16_t *Zf)
{
    const int rows = (n + 127) / 128 * 128;
    k_extract_tc<<<ex_grid(rows, n_dev != nullptr), 128, 0, st>>>(xhat, H, W, anchors, n, rowmap, n_dev, fmt, split,
                                                                  Zhi, Zlo, zz, zsc2, mu, Zf);
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
