// Patch estimation (Eqs. 15-16) on the tensor cores, grouped by component.
//
// For the patches that selected component k (a work item of up to 128):
//   c = Ubar_k^T z,  c'_j = (gamma_kj - gamma_kP) c_j,
//   zhat = Ubar_k c' + gamma_kP z + mu
// as two chained GEMMs in the split BF16 form (hi*hi + lo*hi + hi*lo, the
// same arithmetic as the split selection pass): the CTA copies its patches'
// split operand rows (extracted once per iteration, with the means) into
// shared memory in the 128-byte-swizzled K-major layout, TMA brings Ubar_k
// in both orientations (hi + lo), the first product lands in TMEM, the
// epilogue scales it by the Wiener gains and writes it back over the patch
// rows as the split A operand of the second product, and the second epilogue
// adds the tail term (z from the extracted rows) and the mean and writes the
// patch's 64 estimates (one FP32 row per anchor) for the reprojection.
#include "epll_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

namespace epll {

constexpr int ET_T = 128;           // patches per work item (the MMA's M)
constexpr int ET_THREADS = 256;     // two warps per TMEM lane quarter, each taking 32 of the 64 columns
constexpr int ET_TILE = ET_T * 128;  // 16 KB: [128 rows][64] BF16
constexpr int ET_B = 64 * 128;       // 8 KB: [64 rows][64] BF16
// A hi/lo (overwritten by C' hi/lo), B1 hi/lo, B2 hi/lo, then barriers and per-row scalars
constexpr int ET_SMEM = 1024 + 2 * ET_TILE + 4 * ET_B + 64 + 3 * ET_T * 4 + 64 * 4;

__global__ void __launch_bounds__(ET_THREADS)
k_estimate_tc(const __grid_constant__ CUtensorMap mapU1, const __grid_constant__ CUtensorMap mapU1lo,
              const __grid_constant__ CUtensorMap mapU2, const __grid_constant__ CUtensorMap mapU2lo,
              const int *__restrict__ anchors, const uint4 *__restrict__ Zhi_g, const uint4 *__restrict__ Zlo_g,
              const float *__restrict__ mu_g,
              const int *__restrict__ perm, const int4 *__restrict__ items, const int *__restrict__ roff,
              const int *__restrict__ rk_, Tables tab, float *__restrict__ zrow, int *__restrict__ err)
{
    if ((int)blockIdx.x >= items[0].w) return;
    extern __shared__ __align__(1024) unsigned char et_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)et_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *Ahi = smem, *Alo = Ahi + ET_TILE, *Chi = Ahi, *Clo = Alo;  // C' over A after GEMM 1
    unsigned char *B1hi = Alo + ET_TILE, *B1lo = B1hi + ET_B, *B2hi = B1lo + ET_B, *B2lo = B2hi + ET_B;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(B2lo + ET_B);  // bases, GEMM 1, GEMM 2
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 3);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    float *s_mu = reinterpret_cast<float *>(bars + 8);
    int *s_anchor = reinterpret_cast<int *>(s_mu + ET_T), *s_patch = s_anchor + ET_T;
    float *s_gw = reinterpret_cast<float *>(s_patch + ET_T);  // Wiener gains of the component (0 beyond r)
    const int4 it = items[1 + blockIdx.x];
    const int k = it.x, first = it.y, cnt_p = it.z;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int o = roff[k], r = rk_[k];
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        for (int b = 0; b < 3; ++b) mbar_init(smem_u32(&bars[b]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    if (threadIdx.x == 0) {
        // B1: rows o..o+63 of the [Rtot][64] copy (GEMM 1: N = basis column, K = pixel);
        // B2: columns o..o+63 of the [64][Rtot] copy (GEMM 2: N = pixel, K = basis column)
        const uint32_t b = smem_u32(&bars[0]);
        mbar_expect_tx(b, 4 * ET_B);
        tma_load_2d(smem_u32(B1hi), &mapU1, 0, o, b);
        tma_load_2d(smem_u32(B1lo), &mapU1lo, 0, o, b);
        tma_load_2d(smem_u32(B2hi), &mapU2, o, 0, b);
        tma_load_2d(smem_u32(B2lo), &mapU2lo, o, 0, b);
    }
    if (threadIdx.x < cnt_p) {
        const int i = perm[first + threadIdx.x];
        s_patch[threadIdx.x] = i;
        s_anchor[threadIdx.x] = anchors ? anchors[i] : i;
        s_mu[threadIdx.x] = mu_g[i];
    }
    __syncthreads();
    if (threadIdx.x < 64) s_gw[threadIdx.x] = threadIdx.x < r ? tab.gw[o + threadIdx.x] : 0.0f;
    // the patches' split operand rows: eight threads per 128-byte row,
    // 16-byte chunks to their swizzled place (all eight loads in flight)
    {
        constexpr int NU = ET_T * 8 / ET_THREADS;
        uint4 h[NU], l[NU];
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const int q = threadIdx.x + u * ET_THREADS, t = q >> 3, c = q & 7;
            h[u] = l[u] = make_uint4(0, 0, 0, 0);
            if (t < cnt_p) {
                const size_t src = (size_t)s_patch[t] * 8 + c;
                h[u] = Zhi_g[src];
                l[u] = Zlo_g[src];
            }
        }
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const int q = threadIdx.x + u * ET_THREADS, t = q >> 3, c = q & 7;
            const uint32_t o2 = (uint32_t)(t * 128 + ((c ^ (t & 7)) << 4));
            *reinterpret_cast<uint4 *>(Ahi + o2) = h[u];
            *reinterpret_cast<uint4 *>(Alo + o2) = l[u];
        }
    }
    fence_proxy_async();
    __syncthreads();
    const uint32_t idesc = idesc_f16(ET_T, 64, 1);
    if (threadIdx.x == 0) {
        if (mbar_wait(smem_u32(&bars[0]), 0, abort_flag)) {
            tc_fence_after();
            const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(B1hi), bl = smem_u32(B1lo);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t q = 32 * kk;
                mma_f16(tbase, sdesc_sw128(ah + q), sdesc_sw128(bh + q), idesc, kk ? 1u : 0u);
                mma_f16(tbase, sdesc_sw128(al + q), sdesc_sw128(bh + q), idesc, 1u);
                mma_f16(tbase, sdesc_sw128(ah + q), sdesc_sw128(bl + q), idesc, 1u);
            }
            mma_commit(smem_u32(&bars[1]));
        }
    }
    __syncwarp();
    // tcgen05.ld is warp-collective: every lane takes the same branch
    bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&bars[1]), 0, abort_flag));
    tc_fence_after();
    // warp w: TMEM lane quarter w % 4 (rows 32 (w % 4) ..), columns 32 (w / 4) .. + 31
    const int qd = warp & 3, hh = warp >> 2;
    const int t = 32 * qd + lane;
    const uint32_t tl = tbase + ((uint32_t)(32 * qd) << 16);
    if (ok) {
        // c'_j = gw_kj c_j (zero beyond the rank), split into the A operand of GEMM 2
        uint32_t c[32];
        tmem_ld_all<32>(tl + (uint32_t)(32 * hh), c);
#pragma unroll
        for (int jl = 0; jl < 4; ++jl) {
            const int j8 = 4 * hh + jl;
            uint32_t ph[4], pl[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 8 * j8 + 2 * q, jc = 8 * jl + 2 * q;
                const float v0 = s_gw[j] * __uint_as_float(c[jc]);
                const float v1 = s_gw[j + 1] * __uint_as_float(c[jc + 1]);
                const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
                ph[q] = *reinterpret_cast<const uint32_t *>(&h);
                pl[q] = *reinterpret_cast<const uint32_t *>(&l);
            }
            const uint32_t off = (uint32_t)(t * 128 + ((j8 ^ (t & 7)) << 4));
            *reinterpret_cast<uint4 *>(Chi + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
            *reinterpret_cast<uint4 *>(Clo + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
        }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && ok) {
        tc_fence_after();
        const uint32_t ah = smem_u32(Chi), al = smem_u32(Clo), bh = smem_u32(B2hi), bl = smem_u32(B2lo);
        const int ksteps = (r + 15) >> 4;
        for (int kk = 0; kk < ksteps; ++kk) {
            const uint32_t q = 32 * kk;
            mma_f16(tbase + 64, sdesc_sw128(ah + q), sdesc_sw128(bh + q), idesc, kk ? 1u : 0u);
            mma_f16(tbase + 64, sdesc_sw128(al + q), sdesc_sw128(bh + q), idesc, 1u);
            mma_f16(tbase + 64, sdesc_sw128(ah + q), sdesc_sw128(bl + q), idesc, 1u);
        }
        mma_commit(smem_u32(&bars[2]));
    }
    __syncwarp();
    ok = __all_sync(0xffffffffu, ok && mbar_wait(smem_u32(&bars[2]), 0, abort_flag));
    tc_fence_after();
    uint32_t v[32];
    if (ok) tmem_ld_all<32>(tl + 64 + (uint32_t)(32 * hh), v);  // whole warp, before the per-row test
    if (ok && t < cnt_p) {
        // zhat = Ubar c' + gamma_P z + mu, z = hi + lo of this row (elements 32 hh .. 32 hh + 31)
        const float gp = tab.gp[k], mu = s_mu[t];
        float4 *dst = reinterpret_cast<float4 *>(zrow + (size_t)s_anchor[t] * PD);
        const size_t zr = (size_t)s_patch[t] * 8;
        uint4 zhs[4], zls[4];
#pragma unroll
        for (int el = 0; el < 4; ++el) {
            zhs[el] = Zhi_g[zr + 4 * hh + el];
            zls[el] = Zlo_g[zr + 4 * hh + el];
        }
#pragma unroll
        for (int el = 0; el < 4; ++el) {
            const int e8 = 4 * hh + el;
            const uint4 zh = zhs[el];
            const uint4 zl = zls[el];
            const uint32_t hw[4] = {zh.x, zh.y, zh.z, zh.w}, lw[4] = {zl.x, zl.y, zl.z, zl.w};
            float out[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&hw[q]);
                const __nv_bfloat162 l = *reinterpret_cast<const __nv_bfloat162 *>(&lw[q]);
                const float z0 = __low2float(h) + __low2float(l), z1 = __high2float(h) + __high2float(l);
                out[2 * q] = fmaf(gp, z0, __uint_as_float(v[8 * el + 2 * q])) + mu;
                out[2 * q + 1] = fmaf(gp, z1, __uint_as_float(v[8 * el + 2 * q + 1])) + mu;
            }
            dst[2 * e8] = make_float4(out[0], out[1], out[2], out[3]);
            dst[2 * e8 + 1] = make_float4(out[4], out[5], out[6], out[7]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tbase) : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(err, 1);
}

epll_status launch_estimate_tc(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                               bool reuse, cudaStream_t st)
{
    Workspace &ws = g->ws;
    epll_status s;
    // split operands and means of every patch (unless the selection left them)
    if (!reuse && (s = launch_extract_split(g, xhat, H, W, anchors, n, st))) return s;
    if ((s = group_by_component(g, ws.kstar, n, ws.perm, ws.items, st))) return s;
    static bool attr = false;
    if (!attr) {
        EPLL_CU(cudaFuncSetAttribute(k_estimate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, ET_SMEM));
        attr = true;
    }
    const size_t R = (size_t)g->Rtot;
    CUtensorMap u1, u1lo, u2, u2lo;
    if ((s = make_map(&u1, g->d_Ub, g->Rtot, 64))) return s;
    if ((s = make_map(&u1lo, g->d_Ub + R * PD, g->Rtot, 64))) return s;
    if ((s = make_map_wide(&u2, g->d_U2b, PD, 64, g->Rtot))) return s;
    if ((s = make_map_wide(&u2lo, g->d_U2b + R * PD, PD, 64, g->Rtot))) return s;
    const int max_items = (n + ET_T - 1) / ET_T + g->K;
    const uint4 *zh = reinterpret_cast<const uint4 *>(ws.Zb);
    const uint4 *zl = reinterpret_cast<const uint4 *>(ws.Zb + ws.zrows * PD);
    k_estimate_tc<<<max_items, ET_THREADS, ET_SMEM, st>>>(u1, u1lo, u2, u2lo, anchors, zh, zl, ws.mu, ws.perm, ws.items,
                                                    g->d_roff, g->d_r, g->tab, ws.zrow, cnt(g, CNT_ERR));
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

}  // namespace epll
