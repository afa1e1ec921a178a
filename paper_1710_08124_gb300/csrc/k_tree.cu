// Gaussian selection down the balanced search tree (Sec. "Speed-up via a
// balanced search tree"): every patch starts at the root and, level after
// level, moves to the child whose flat-tailed Gaussian (the same score as
// Eq. 14, on the node's own tables) is cheapest, until it reaches a leaf,
// i.e. a component of the model.
//
// The DC-free patches are extracted once per iteration as split BF16
// operands (hi + lo) with their |z|^2; then one launch per level.  The
// patches are grouped by their current node (the counting sort of the
// estimation step, keyed by node), and a CTA takes one group of up to 128
// patches of one node: it copies their operand rows into shared memory
// (128-byte-swizzled K-major rows), loads the children's concatenated scaled
// bases (consecutive in the node model's column order, at most 256 columns)
// by TMA, accumulates hi*hi + lo*hi + hi*lo into TMEM and scores each child
// in the epilogue.  Ties go to the lowest child.  The smallest top-2 gap met
// on the way is kept per patch.
#include "epll_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

#include <cfloat>

namespace epll {

constexpr int TL_T = 128;
constexpr int TL_TILE = TL_T * 128;  // 16 KB: [128 rows][64] BF16
constexpr int TL_BMAX = 256;         // basis columns of one node's children
constexpr int TL_B = TL_BMAX * 128;  // 32 KB
constexpr int TL_CH = 4;             // children of one node
constexpr int TL_SMEM = 1024 + 2 * TL_TILE + 2 * TL_B + 64 + 2 * TL_T * 4;

__global__ void __launch_bounds__(TL_T)
k_tree_level(const __grid_constant__ CUtensorMap mapBs, const __grid_constant__ CUtensorMap mapBlo,
             const uint4 *__restrict__ Zhi, const uint4 *__restrict__ Zlo, const float *__restrict__ zz,
             const int *__restrict__ perm, const int4 *__restrict__ items, const int *__restrict__ child,
             const int *__restrict__ leaf, const int *__restrict__ roff, const int *__restrict__ rk_, Tables tab,
             int first_level, int last_level,
             int *__restrict__ node, int *__restrict__ kstar, float *__restrict__ gap, int *__restrict__ err)
{
    if ((int)blockIdx.x >= items[0].w) return;
    extern __shared__ __align__(1024) unsigned char tl_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)tl_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *Ahi = smem, *Alo = Ahi + TL_TILE, *Bhi = Alo + TL_TILE, *Blo = Bhi + TL_B;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(Blo + TL_B);  // bases, MMA
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    float *s_zz = reinterpret_cast<float *>(bars + 8);
    int *s_patch = reinterpret_cast<int *>(s_zz + TL_T);
    const int4 it = items[1 + blockIdx.x];
    const int v = it.x, first = it.y, cnt_p = it.z;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = child[v], c1 = child[v + 1];
    // the children's columns: from the first child's offset to the end of the
    // last child's rank (padded to 8; the node model's trailing padding excluded)
    const int col0 = roff[c0], ncols = roff[c1 - 1] + ((rk_[c1 - 1] + 7) & ~7) - col0;
    const int nbox = (ncols + 63) >> 6, nmma = (ncols + 15) & ~15;
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
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
    const uint32_t tbase = *tslot;
    if (threadIdx.x == 0) {
        const uint32_t b = smem_u32(&bars[0]);
        mbar_expect_tx(b, 2 * nbox * 64 * 128);
        for (int q = 0; q < nbox; ++q) {
            tma_load_2d(smem_u32(Bhi + q * 64 * 128), &mapBs, 0, col0 + 64 * q, b);
            tma_load_2d(smem_u32(Blo + q * 64 * 128), &mapBlo, 0, col0 + 64 * q, b);
        }
    }
    if (threadIdx.x < cnt_p) {
        const int i = perm[first + threadIdx.x];
        s_patch[threadIdx.x] = i;
        s_zz[threadIdx.x] = zz[i];
    }
    __syncthreads();
    // the group's rows of the split operands extracted once per iteration:
    // eight threads per 128-byte row, 16-byte chunks to their swizzled place
    for (int q = threadIdx.x; q < TL_T * 8; q += TL_T) {
        const int t = q >> 3, c = q & 7;
        uint4 h = make_uint4(0, 0, 0, 0), l = make_uint4(0, 0, 0, 0);
        if (t < cnt_p) {
            const size_t src = (size_t)s_patch[t] * 8 + c;
            h = Zhi[src];
            l = Zlo[src];
        }
        const uint32_t o = (uint32_t)(t * 128 + ((c ^ (t & 7)) << 4));
        *reinterpret_cast<uint4 *>(Ahi + o) = h;
        *reinterpret_cast<uint4 *>(Alo + o) = l;
    }
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (mbar_wait(smem_u32(&bars[0]), 0, abort_flag)) {
            tc_fence_after();
            const uint32_t idesc = idesc_f16(TL_T, nmma, 1);
            const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
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
    const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&bars[1]), 0, abort_flag));
    tc_fence_after();
    if (ok) {
        // per child: sum of squared scaled projections over its columns
        int bound[TL_CH + 1];
        const int nch = c1 - c0;
#pragma unroll
        for (int q = 0; q <= TL_CH; ++q) bound[q] = q < nch ? roff[c0 + q] - col0 : ncols;
        float part[TL_CH] = {0.0f, 0.0f, 0.0f, 0.0f};
        const uint32_t tl = tbase + ((uint32_t)(32 * warp) << 16);
        for (int cb = 0; cb < nmma; cb += 32) {
            uint32_t r[32];
            tmem_ld32(tl + (uint32_t)cb, r);
            tmem_wait(r);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int col = cb + q;
                const float c = __uint_as_float(r[q]);
                const float c2 = col < ncols ? c * c : 0.0f;
#pragma unroll
                for (int u = 0; u < TL_CH; ++u)
                    if (col >= bound[u] && col < bound[u + 1]) part[u] += c2;
            }
        }
        const int t = 32 * warp + lane;
        if (t < cnt_p) {
            const float zz = s_zz[t];
            float s1 = FLT_MAX, s2 = FLT_MAX;
            int best = c0;
#pragma unroll
            for (int u = 0; u < TL_CH; ++u) {
                if (u < nch) {
                    const int c = c0 + u;
                    const float sc = tab.cst_hi[c] + tab.t_hi[c] * zz + tab.sgn[c] * part[u];
                    if (sc < s1) {
                        s2 = s1;
                        s1 = sc;
                        best = c;
                    } else if (sc < s2) {
                        s2 = sc;
                    }
                }
            }
            const int i = s_patch[t];
            const float g = nch > 1 ? s2 - s1 : FLT_MAX;
            gap[i] = first_level ? g : fminf(gap[i], g);
            if (last_level) kstar[i] = leaf[best];
            else node[i] = best;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tbase) : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(err, 1);
}

static epll_status ensure_tree_ws(epll_gmm *g)
{
    Workspace &ws = g->ws;
    const TreeState *tr = g->tree;
    if (ws.tnode && ws.tree_cap >= ws.capN && ws.tree_nodes >= tr->n_nodes) return EPLL_OK;
    void *ptrs[] = {ws.tnode, ws.tcounts, ws.titems};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    ws.tnode = nullptr;
    ws.tcounts = nullptr;
    ws.titems = nullptr;
    const size_t N = ws.capN;
    cudaError_t e = cudaSuccess;
    auto A = [&](void **q, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(q, bytes); };
    A((void **)&ws.tnode, N * sizeof(int));
    A((void **)&ws.tcounts, (size_t)tr->n_nodes * sizeof(int));
    A((void **)&ws.titems, (2 + N / 128 + (size_t)tr->n_nodes) * sizeof(int4));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(EPLL_ENOMEM, std::string("tree workspace: ") + cudaGetErrorString(e));
    }
    ws.tree_cap = N;
    ws.tree_nodes = tr->n_nodes;
    return EPLL_OK;
}

epll_status launch_select_tree(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                               cudaStream_t st)
{
    Workspace &ws = g->ws;
    const TreeState *tr = g->tree;
    epll_gmm *tm = tr->tm;
    epll_status s;
    if ((s = ensure_tree_ws(g))) return s;
    static bool attr = false;
    if (!attr) {
        EPLL_CU(cudaFuncSetAttribute(k_tree_level, cudaFuncAttributeMaxDynamicSharedMemorySize, TL_SMEM));
        attr = true;
    }
    CUtensorMap bs, bslo;
    if ((s = make_map(&bs, tm->tab.Bs, tm->Rtot, 64))) return s;
    if ((s = make_map(&bslo, tm->tab.Bs_lo, tm->Rtot, 64))) return s;
    // split BF16 DC-free patches and |z|^2, once for every level
    if ((s = launch_extract_split(g, xhat, H, W, anchors, n, st))) return s;
    EPLL_CU(cudaMemsetAsync(ws.tnode, 0, sizeof(int) * (size_t)n, st));  // every patch at the root
    EPLL_CU(cudaMemsetAsync(cnt(g, CNT_NFLAG), 0, sizeof(int), st));     // no near-tie list
    const int max_items = (n + TL_T - 1) / TL_T + tr->n_nodes;
    for (int lev = 0; lev < tr->depth; ++lev) {
        if ((s = group_by_key(g, ws.tnode, n, tr->n_nodes, ws.tcounts, ws.perm, ws.titems, st))) return s;
        const int last = lev == tr->depth - 1;
        prof_begin(g, st);
        k_tree_level<<<max_items, TL_T, TL_SMEM, st>>>(bs, bslo, reinterpret_cast<const uint4 *>(ws.Zb),
                                                       reinterpret_cast<const uint4 *>(ws.Zb + ws.zrows * PD),
                                                       ws.zz, ws.perm, ws.titems,
                                                       tr->d_child, tr->d_leaf, tm->d_roff, tm->d_r, tm->tab, lev == 0,
                                                       last, ws.tnode, ws.kstar, ws.gap, cnt(g, CNT_ERR));
        prof_end(g, st, n, 2.0 * PD * (double)tr->child_cols_mean);
        EPLL_LAUNCHED(g);
    }
    return EPLL_OK;
}

}  // namespace epll
