// Patch estimation (Eqs. 15-16) on the tensor cores, grouped by component.
//
// For the patches that selected component k (a work item of up to 128):
//   c = Ubar_k^T z,  c'_j = (gamma_kj - gamma_kP) c_j,
//   zhat = Ubar_k c' + gamma_kP z + mu
// as two chained GEMMs in the split BF16 form (hi*hi + lo*hi + hi*lo, the
// same arithmetic as the split selection pass).
//
// One persistent CTA per SM walks the work items, two in flight, one per
// stage s in {0, 1}; each stage has its own producer warps, MMA thread and
// epilogue warps:
//   - a producer warp copies an item's split operand rows (extracted once
//     per iteration, with the means) into the stage in the 128-byte-swizzled
//     K-major layout with cp.async, and TMA brings Ubar_k in both
//     orientations (hi + lo); the item's indices and scalars are read while
//     the stage is still in use;
//   - the MMA thread issues the first product into the stage's TMEM columns,
//     then, once the epilogue prepared its operands, the second product
//     accumulating onto the tail term; the second product's completion
//     frees the stage's shared memory for the item after next;
//   - eight epilogue warps scale the first product by the Wiener gains into
//     the split A operand of the second product (over the patch rows, which
//     they read first), store gamma_kP z + mu into the second product's
//     accumulator columns, and after the second product write the patch's 64
//     estimates for the reprojection (eight 32-byte patch-row segments,
//     segment u into plane u of the estimate buffer at the patch's index in
//     the subset, and that index at the patch's anchor) while the producers
//     already fill the stage again.
// Every wait is bounded; a timeout reaches the host as an error.
#include "epll_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace epll {

constexpr int ET_T = 128;                     // patches per work item (the MMA's M)
constexpr int ET_TILE = ET_T * 128;           // 16 KB: [128 rows][64] BF16
constexpr int ET_B = 64 * 128;                // 8 KB: [64 rows][64] BF16
constexpr int ET_STAGE = 2 * ET_TILE + 4 * ET_B;  // A hi, A lo (then C' hi, lo), B1 hi, B1 lo, B2 hi, B2 lo
constexpr int ET_PROD = 1;                    // producer warp per stage (four rows per lane)
constexpr int ET_EPI = 8;                     // epilogue warps per stage (two per TMEM lane quarter)
constexpr int ET_WARPS = 2 + 2 * ET_PROD + 2 * ET_EPI;  // MMA warps, producers, epilogues
constexpr int ET_THREADS = 32 * ET_WARPS;

struct EtStage {  // an item's scalars, beside its stage
    int anchor[ET_T];
    int patch[ET_T];  // index in the subset
    float mu[ET_T];
    float gw[64];  // Wiener gains of the component (0 beyond the rank)
    int r, cnt;
    float gp;
    int pad;
};
// barriers per stage: full, mma1, cprep, mma2
constexpr int ET_STG = 40;  // floats per row of an epilogue warp's staging tile (32 rows x 32 values)
constexpr int ET_SMEM = 1024 + 2 * ET_STAGE + 2 * (int)sizeof(EtStage) + 8 * 8 + 16 + 2 * ET_EPI * 32 * ET_STG * 4;

// 96 registers: the register file is split between the SM's four sub-partitions,
// each holding at most five of the 20 warps (5 x 32 x 96 <= 16384)
__global__ void __maxnreg__(96)
k_estimate_tc(const __grid_constant__ CUtensorMap mapU1, const __grid_constant__ CUtensorMap mapU1lo,
              const __grid_constant__ CUtensorMap mapU2, const __grid_constant__ CUtensorMap mapU2lo,
              const uint4 *__restrict__ Zhi_g, const uint4 *__restrict__ Zlo_g,
              const int *__restrict__ anchors, const float *__restrict__ mu_g,
              const int *__restrict__ perm, const int4 *__restrict__ items, const int *__restrict__ roff,
              const int *__restrict__ rk_, Tables tab, float *__restrict__ zrow, int *__restrict__ inv,
              long long npix, int *__restrict__ err)
{
    pdl_enter();
    extern __shared__ __align__(1024) unsigned char et_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)et_raw + 1023) & ~(uintptr_t)1023);
    EtStage *sc = reinterpret_cast<EtStage *>(smem + 2 * ET_STAGE);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(sc + 2);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    float *stg_all = reinterpret_cast<float *>(tslot + 4);  // epilogue warps' staging tiles
    const uint32_t bar0 = smem_u32(bars);
#define ET_FULL(s) (bar0 + 8u * (uint32_t)(s))
#define ET_MMA1(s) (bar0 + 8u * (uint32_t)(2 + (s)))
#define ET_CPREP(s) (bar0 + 8u * (uint32_t)(4 + (s)))
#define ET_MMA2(s) (bar0 + 8u * (uint32_t)(6 + (s)))
#define ET_STAGE_PTR(s) (smem + (s) * ET_STAGE)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_items = items[0].w;
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        for (int s = 0; s < 2; ++s) {
            mbar_init(ET_FULL(s), 32 * ET_PROD + 1);  // producer threads + the arrival that sets the TMA byte count
            mbar_init(ET_MMA1(s), 1);
            mbar_init(ET_CPREP(s), 32 * ET_EPI);
            mbar_init(ET_MMA2(s), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;  // stage s: columns 128 s (first product) and 128 s + 64 (second)
    const uint32_t idesc = idesc_f16(ET_T, 64, 1);
    // the j-th item of this CTA is item blockIdx.x + j gridDim.x, on stage j % 2;
    // each stage's barriers complete once per item of the stage, parity (j / 2) % 2

    if (warp < 2) {
        // ---------------------------------------------------------------- MMA issue, stage `warp`
        const int s = warp;
        if (lane == 0) {
            const uint32_t ah = smem_u32(ET_STAGE_PTR(s)), al = ah + ET_TILE;
            const uint32_t b1h = ah + 2 * ET_TILE, b1l = b1h + ET_B, b2h = b1l + ET_B, b2l = b2h + ET_B;
            const uint32_t d1 = tbase + 128 * s, d2 = d1 + 64;
            for (int j = s; (int)blockIdx.x + j * (int)gridDim.x < n_items; j += 2) {
                const uint32_t ph = (j >> 1) & 1;
                if (!mbar_wait(ET_FULL(s), ph, abort_flag)) break;
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t q = 32 * kk;
                    mma_f16(d1, sdesc_sw128(ah + q), sdesc_sw128(b1h + q), idesc, kk ? 1u : 0u);
                    mma_f16(d1, sdesc_sw128(al + q), sdesc_sw128(b1h + q), idesc, 1u);
                    mma_f16(d1, sdesc_sw128(ah + q), sdesc_sw128(b1l + q), idesc, 1u);
                }
                mma_commit(ET_MMA1(s));
                // second product onto the tail term the epilogue stored in d2,
                // A = C' (written over the patch rows)
                const int ksteps = (sc[s].r + 15) >> 4;
                if (!mbar_wait(ET_CPREP(s), ph, abort_flag)) break;
                tc_fence_after();
                for (int kk = 0; kk < ksteps; ++kk) {
                    const uint32_t q = 32 * kk;
                    mma_f16(d2, sdesc_sw128(ah + q), sdesc_sw128(b2h + q), idesc, 1u);
                    mma_f16(d2, sdesc_sw128(al + q), sdesc_sw128(b2h + q), idesc, 1u);
                    mma_f16(d2, sdesc_sw128(ah + q), sdesc_sw128(b2l + q), idesc, 1u);
                }
                mma_commit(ET_MMA2(s));
            }
        }
        __syncwarp();
    } else if (warp < 2 + 2 * ET_PROD) {
        // ---------------------------------------------------------------- producers of stage s
        const int s = (warp - 2) / ET_PROD;
        const int p = (warp - 2 - s * ET_PROD) * 32 + lane;  // rows p, p + 32, p + 64, p + 96
        constexpr int NR = ET_T / (32 * ET_PROD);
        EtStage &st = sc[s];
        unsigned char *A = ET_STAGE_PTR(s);
        const uint32_t a0 = smem_u32(A);
        for (int j = s; (int)blockIdx.x + j * (int)gridDim.x < n_items; j += 2) {
            // the item's indices and scalars, read while the stage is still in use
            const int4 it = items[1 + (int)blockIdx.x + j * (int)gridDim.x];
            const int k = it.x, first = it.y, cnt = it.z;
            int row[NR], anc[NR];
            float mu[NR];
#pragma unroll
            for (int h = 0; h < NR; ++h) row[h] = p + 32 * h < cnt ? perm[first + p + 32 * h] : -1;
            const int o = roff[k], r = rk_[k];
            const float gw0 = p < r ? tab.gw[o + p] : 0.0f, gw1 = p + 32 < r ? tab.gw[o + p + 32] : 0.0f;
            const float gp = tab.gp[k];
#pragma unroll
            for (int h = 0; h < NR; ++h) {
                anc[h] = 0;
                mu[h] = 0.0f;
                if (row[h] >= 0) {
                    anc[h] = anchors ? anchors[row[h]] : row[h];
                    mu[h] = mu_g[row[h]];
                }
            }
            // the second product of the stage's previous item (j - 2) has read the stage
            if (j >= 2 && !__all_sync(0xffffffffu, mbar_wait(ET_MMA2(s), ((j >> 1) - 1) & 1, abort_flag))) break;
            if (p == 0) {
                st.r = r;
                st.cnt = cnt;
                st.gp = gp;
                // B1: rows o..o+63 of the [Rtot][64] copy (first product: N = basis column, K = pixel);
                // B2: columns o..o+63 of the [64][Rtot] copy (second product: N = pixel, K = basis column)
                const uint32_t b = ET_FULL(s), bb = a0 + 2 * ET_TILE;
                mbar_expect_tx(b, 4 * ET_B);
                tma_load_2d(bb, &mapU1, 0, o, b);
                tma_load_2d(bb + ET_B, &mapU1lo, 0, o, b);
                tma_load_2d(bb + 2 * ET_B, &mapU2, o, 0, b);
                tma_load_2d(bb + 3 * ET_B, &mapU2lo, o, 0, b);
            }
            st.gw[p] = gw0;
            st.gw[p + 32] = gw1;
#pragma unroll
            for (int h = 0; h < NR; ++h) {
                st.anchor[p + 32 * h] = anc[h];
                st.patch[p + 32 * h] = row[h];
                st.mu[p + 32 * h] = mu[h];
            }
            // the rows' split operands straight to their swizzled places (cp.async):
            // eight lanes per row, one 16-byte chunk each, so a warp instruction
            // covers four whole rows; rows past the count are zeros
            const int c = lane & 7;
#pragma unroll
            for (int m = 0; m < ET_T / 4; ++m) {
                const int q = 4 * m + (lane >> 3);
                const int i = __shfl_sync(0xffffffffu, row[m >> 3], q & 31);  // row q is held by lane q % 32
                const uint32_t o2 = a0 + (uint32_t)(q * 128 + ((c ^ (q & 7)) << 4));
                if (i >= 0) {
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(o2), "l"(Zhi_g + (size_t)i * 8 + c)
                                 : "memory");
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(o2 + ET_TILE),
                                 "l"(Zlo_g + (size_t)i * 8 + c)
                                 : "memory");
                } else {
                    *reinterpret_cast<uint4 *>(A + q * 128 + (c << 4)) = make_uint4(0, 0, 0, 0);
                    *reinterpret_cast<uint4 *>(A + ET_TILE + q * 128 + (c << 4)) = make_uint4(0, 0, 0, 0);
                }
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            fence_proxy_async();
            mbar_arrive(ET_FULL(s));
        }
    } else {
        // ---------------------------------------------------------------- epilogue of stage s
        const int ew = warp - 2 - 2 * ET_PROD;
        const int s = ew / ET_EPI;
        const int qd = warp & 3;                // the TMEM lane quarter this warp may access
        const int hh = (ew % ET_EPI) >> 2;      // columns 32 hh .. 32 hh + 31
        const int t = 32 * qd + lane;           // patch row
        const uint32_t tl = tbase + ((uint32_t)(32 * qd) << 16) + 128 * s + 32 * hh;
        unsigned char *A = ET_STAGE_PTR(s);
        const EtStage &st = sc[s];
        float *stg = stg_all + ew * 32 * ET_STG;
        for (int j = s; (int)blockIdx.x + j * (int)gridDim.x < n_items; j += 2) {
            const uint32_t ph = (j >> 1) & 1;
            // tcgen05.ld is warp-collective: every lane takes the same branch
            bool ok = __all_sync(0xffffffffu, mbar_wait(ET_FULL(s), ph, abort_flag));
            ok = ok && __all_sync(0xffffffffu, mbar_wait(ET_MMA1(s), ph, abort_flag));
            if (!ok) break;
            tc_fence_after();
            // the row's destination, read before the stage is handed back
            const int cnt_item = st.cnt;
            const bool live = t < cnt_item;
            const int pi = st.patch[t];
            if (live && hh == 0) inv[st.anchor[t]] = pi;
            {
                // c'_j = gw_kj c_j (zero beyond the rank) split into the A operand of the
                // second product, written over this thread's own part of the patch row,
                // which first gives the tail term gamma_P z + mu
                const float gp = st.gp, mu = st.mu[t];
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    uint32_t c[16];  // the first product, replaced column by column by the tail term
                    tmem_ld16_wait(tl + 16 * half, c);
#pragma unroll
                    for (int jl = 0; jl < 2; ++jl) {
                        const int j8 = 4 * hh + 2 * half + jl;
                        const uint32_t off = (uint32_t)(t * 128 + ((j8 ^ (t & 7)) << 4));
                        const uint4 zh = *reinterpret_cast<const uint4 *>(A + off);
                        const uint4 zl = *reinterpret_cast<const uint4 *>(A + ET_TILE + off);
                        const uint32_t hw[4] = {zh.x, zh.y, zh.z, zh.w}, lw[4] = {zl.x, zl.y, zl.z, zl.w};
                        uint32_t ph2[4], pl[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162 *>(&hw[q]);
                            const __nv_bfloat162 lb = *reinterpret_cast<const __nv_bfloat162 *>(&lw[q]);
                            const float z0 = __low2float(hb) + __low2float(lb);
                            const float z1 = __high2float(hb) + __high2float(lb);
                            const int jj = 8 * j8 + 2 * q, jc = 8 * jl + 2 * q;
                            const float v0 = st.gw[jj] * __uint_as_float(c[jc]);
                            const float v1 = st.gw[jj + 1] * __uint_as_float(c[jc + 1]);
                            c[jc] = __float_as_uint(fmaf(gp, z0, mu));
                            c[jc + 1] = __float_as_uint(fmaf(gp, z1, mu));
                            const __nv_bfloat162 hv = __floats2bfloat162_rn(v0, v1);
                            const __nv_bfloat162 lv =
                                __floats2bfloat162_rn(v0 - __low2float(hv), v1 - __high2float(hv));
                            ph2[q] = *reinterpret_cast<const uint32_t *>(&hv);
                            pl[q] = *reinterpret_cast<const uint32_t *>(&lv);
                        }
                        *reinterpret_cast<uint4 *>(A + off) = make_uint4(ph2[0], ph2[1], ph2[2], ph2[3]);
                        *reinterpret_cast<uint4 *>(A + ET_TILE + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
                    }
                    tmem_st16(tl + 64 + 16 * half, c);
                }
                tmem_wait_st();
            }
            fence_proxy_async();
            tc_fence_before();
            mbar_arrive(ET_CPREP(s));
            ok = __all_sync(0xffffffffu, mbar_wait(ET_MMA2(s), ph, abort_flag));
            if (!ok) break;
            tc_fence_after();
            // the warp's 32 rows x 32 estimates (patch rows 4 hh .. 4 hh + 3) through its
            // staging tile, then written two lanes per 32-byte segment: a store
            // instruction covers sixteen whole segments of one plane
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                uint32_t v[16];
                tmem_ld16_wait(tl + 64 + 16 * half, v);  // whole warp
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    *reinterpret_cast<uint4 *>(stg + lane * ET_STG + 16 * half + 4 * q) =
                        make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
            __syncwarp();
            {
                const int cntw = cnt_item - 32 * qd;  // live rows of this warp
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int rr = 16 * h2 + (lane >> 1), part = lane & 1;
                    const int prow = __shfl_sync(0xffffffffu, pi, rr);
#pragma unroll
                    for (int el = 0; el < 4; ++el) {
                        const float4 val = *reinterpret_cast<const float4 *>(stg + rr * ET_STG + 8 * el + 4 * part);
                        if (rr < cntw)
                            *reinterpret_cast<float4 *>(zrow + ((size_t)(4 * hh + el) * npix + prow) * PS + 4 * part) = val;
                    }
                }
            }
            __syncwarp();  // the staging tile is rewritten by the next item
            // the next item's first epilogue writes the tail term into these columns
            tc_fence_before();
            __syncwarp();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tbase) : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(err, 1);
#undef ET_FULL
#undef ET_MMA1
#undef ET_CPREP
#undef ET_MMA2
#undef ET_STAGE_PTR
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
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        EPLL_CU(cudaGetDevice(&dev));
        EPLL_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int max_items = (n + ET_T - 1) / ET_T + g->K;
    int grid = max_items < sms ? max_items : sms;
    // a batch lane shares the GPU with the other lanes' kernels: its CTAs
    // (one per SM, which they fill) take three work items each at least
    if (g->lane) {
        const int cap = (max_items + 2) / 3;
        grid = std::max(1, std::min(grid, cap));
    }
    const uint4 *zh = reinterpret_cast<const uint4 *>(ws.Zb);
    const uint4 *zl = reinterpret_cast<const uint4 *>(ws.Zb + ws.zrows * PD);
    EPLL_CU(launch_pdl(k_estimate_tc, dim3(grid), dim3(ET_THREADS), ET_SMEM, st, u1, u1lo, u2, u2lo, zh, zl, anchors, ws.mu, ws.perm, ws.items,
                                                   g->d_roff, g->d_r, g->tab, ws.zrow, ws.inv, (long long)H * W,
                                                   cnt(g, CNT_ERR)));
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

}  // namespace epll
