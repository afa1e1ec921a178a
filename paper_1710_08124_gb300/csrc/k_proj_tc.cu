// Gaussian selection on the 5th-generation tensor cores (tcgen05).
//
// The projection of Eq. 13, C = Z [Ubar_1 ... Ubar_K] (Z: sampled DC-free
// patches, 64 wide), is a dense contraction with a reduction depth of only
// 64.  Each CTA owns 128 patches: their 16-bit tile is loaded once by TMA
// (128-byte swizzle) and stays in shared memory while the basis streams
// through a multi-stage TMA ring.  One thread issues tcgen05.mma into FP32
// accumulators in tensor memory (2-4 buffers, 512 columns); up to sixteen
// epilogue warps (four per TMEM lane quarter, each owning a quarter of the
// columns) read the accumulators back with tcgen05.ld and fold them straight
// into the scores of Eq. 14, keeping the best and second-best component per
// patch, so the K x N score matrix never exists anywhere.
//
// The basis columns are pre-scaled by sqrt|q_kj| (q_kj = 1/nu_kj - 1/nu_kP,
// Eq. 14), so the epilogue needs one FMA per accumulator element:
//   score_k = cst_k + t_k |z|^2 + sign_k * sum_j (sqrt|q_kj| c_kj)^2.
// Operands are BF16 or FP16 (kind::f16, FP32 accumulation); the 3-term
// variant splits both operands into hi + lo BF16 parts and accumulates
// hi*hi + lo*hi + hi*lo, which brings the score error close to FP32.
// Patches whose top-2 gap is below tau_abs + tau_rel |z|^2 max_k(1/nu_min)
// (the error bound of the arithmetic) go to the compensated rescoring.
#include "epll_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cfloat>
#include <climits>
#include <mutex>

namespace epll {

// ---------------------------------------------------------------- main kernel
constexpr int TC_M = 128;
constexpr int TC_SMEM_BUDGET = 200 * 1024;

template <int BN, int NT, int RR, bool CAND = false, bool PAIR = false>
struct TcCfg {
    // NT: 1 one 16-bit product, 3 split BF16 (three products), 8 one E4M3 product
    // PAIR: a CTA pair shares each MMA (M = 256); each CTA holds its own 128
    // patch rows and half of every basis tile
    static constexpr int ROWB = NT == 8 ? 64 : 128;            // bytes per 64-element row
    static constexpr int A_TILE = TC_M * ROWB;
    static constexpr int A_BYTES = A_TILE * (NT == 3 ? 2 : 1); // one A buffer (hi [+ lo])
    static constexpr int B_ROWS = PAIR ? BN / 2 : BN;          // basis rows this CTA loads per tile
    static constexpr int B_TILE = B_ROWS * ROWB;
    static constexpr int B_STAGE = B_TILE * (NT == 3 ? 2 : 1);
    static constexpr int STAGES_RAW = (TC_SMEM_BUDGET - 2 * A_BYTES) / B_STAGE;
    static constexpr int STAGES = STAGES_RAW > 8 ? 8 : STAGES_RAW;
    static constexpr int NB = 512 / BN;                        // TMEM accumulator buffers
    // epilogue column groups: each group (one warp per TMEM lane quarter)
    // owns whole components of BN / NG columns; with ragged ranks the four
    // groups split every tile at component boundaries (the model's columns
    // are laid out so that no component straddles a 256-column tile)
    static constexpr int NG = RR == 0 ? 4 : (BN / RR >= 4 ? 4 : BN / RR);
    static constexpr int EWS = 4 * NG;                         // epilogue warps of one set
    // With four accumulator buffers and at most eight warps to a set, two
    // sets take alternate buffers (each has two tiles' time for one), so the
    // MMA may run three tiles ahead of the slowest warp.
    static constexpr int SETS = (EWS <= 8 && NB >= 4) ? 2 : 1;
    static constexpr int EW = EWS * SETS;                      // epilogue warps
    static constexpr int NP = NG * SETS;                       // partial results per row to merge
    static constexpr int THREADS = 64 + 32 * EW;               // warp 0 TMA, warp 1 MMA, then the epilogue
    static constexpr int COLS = BN / NG;                       // columns per epilogue warp
    static constexpr int MW = CAND ? 8 : 3;                    // merge words per row and part
    static constexpr int CTRL = 1024 + (NP - 1) * TC_M * MW * 4; // barriers + the [NP-1][128][MW] merge buffer
    static constexpr int SMEM = 1024 + 2 * A_BYTES + STAGES * B_STAGE + CTRL;
};

struct TcCtrl {
    unsigned long long a_full[2], a_empty[2];
    unsigned long long b_full[8], b_empty[8];
    unsigned long long t_full[4], t_empty[4];
    unsigned long long drain;
    // CTA pairs: rank 1's operand tiles landed (relayed to rank 0's MMA
    // thread), and the end-of-kernel handshake
    unsigned long long ap_full[2], bp_full[8];
    unsigned long long bye;
    uint32_t tmem_base;
    int abort_flag;
};

__device__ __forceinline__ void top2(float s, int k, float &s1, float &s2, int &k1)
{
    if (s < s1) {
        s2 = s1;
        s1 = s;
        k1 = k;
    } else {
        s2 = fminf(s2, s);
    }
}

// (score, component) order: the lower component first among equal scores
__device__ __forceinline__ bool sk_less(float a, int ka, float b, int kb) { return a < b || (a == b && ka < kb); }

// Running four lowest scores of one thread's row, ascending, for components
// that arrive in increasing index order: strict comparisons then keep the
// lower index first among equal scores.  Empty slots hold (FLT_MAX, INT_MAX).
__device__ __forceinline__ void top4_inc(float s, int k, float (&cs)[4], int (&ck)[4])
{
    if (s < cs[3]) {
        if (s < cs[1]) {
            cs[3] = cs[2]; ck[3] = ck[2];
            cs[2] = cs[1]; ck[2] = ck[1];
            if (s < cs[0]) {
                cs[1] = cs[0]; ck[1] = ck[0];
                cs[0] = s; ck[0] = k;
            } else {
                cs[1] = s; ck[1] = k;
            }
        } else if (s < cs[2]) {
            cs[3] = cs[2]; ck[3] = ck[2];
            cs[2] = s; ck[2] = k;
        } else {
            cs[3] = s; ck[3] = k;
        }
    }
}

// The four lowest (score, component) pairs, ascending, for pairs in any
// order (merging the column groups); empty slots hold (FLT_MAX, INT_MAX).
__device__ __forceinline__ void top4(float s, int k, float (&cs)[4], int (&ck)[4])
{
    if (sk_less(s, k, cs[3], ck[3])) {
        cs[3] = s;
        ck[3] = k;
#pragma unroll
        for (int j = 3; j > 0; --j) {
            if (sk_less(cs[j], ck[j], cs[j - 1], ck[j - 1])) {
                const float ts = cs[j]; cs[j] = cs[j - 1]; cs[j - 1] = ts;
                const int tk = ck[j]; ck[j] = ck[j - 1]; ck[j - 1] = tk;
            }
        }
    }
}

// Persistent: CTA b takes the 128-row tiles b, b + gridDim.x, ... of the n
// rows (n read from the device when n_dev is given).  Two A buffers let the
// next tile's patches load while the current tile is multiplied; the basis
// ring and the TMEM accumulator buffers run on across tiles, so the epilogue
// of one tile overlaps the MMAs of the next.
// DUMP = true: instead of the top-2 selection every component's score is
// written to scores[row * K + k]; blockIdx.y then takes a slice of the basis
// tiles (uniform ranks only, so no component straddles two slices).
// CAND = true (one-term first pass): the four best components are kept; a
// patch whose top-2 gap is within the error bound is listed (flag[f] = row)
// with its candidates, the components within that bound of the best, in
// cand[f] (-1: absent); a first candidate of -1 means the band may hold more
// than four components.
// PAIR = true (launched in clusters of two, n given by the host): the two
// CTAs of a cluster take 256-row tiles together, rank r the rows
// 128 r .. 128 r + 127 of each and the basis rows BN/2 r .. BN/2 r + BN/2 - 1
// of each basis tile.  Rank 0's MMA thread issues cta_group::2 MMAs
// (M = 256) once both CTAs' tiles have landed (rank 1's warp 1 relays its
// TMA completions), and its commits arrive on the barriers of both CTAs; the
// epilogue warps of both hand each accumulator buffer back to rank 0.  Each
// SM thus streams half of every basis tile through its shared memory.
template <int BN, int NT, int RR, bool DUMP, bool CAND, bool PAIR = false>
__global__ void __launch_bounds__(TcCfg<BN, NT, RR, CAND, PAIR>::THREADS, 1)
k_proj_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapAlo,
          const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapBlo,
          int n, const int *__restrict__ rowmap, const int *__restrict__ n_dev, int K, int Rtot,
          uint32_t idesc, const float *__restrict__ zz, const int *__restrict__ colk,
          const int4 *__restrict__ tileg, Tables tab,
          float tau_abs, float tau_rel, int *__restrict__ kstar, float *__restrict__ gap,
          int *__restrict__ flag, int *__restrict__ nflag, int *__restrict__ err,
          float *__restrict__ scores, const float *__restrict__ zsc2, int4 *__restrict__ cand)
{
    using C = TcCfg<BN, NT, RR, CAND, PAIR>;
    static_assert(!(DUMP && CAND), "one output form");
    static_assert(!PAIR || (!DUMP && NT != 8), "CTA pairs: first pass, 16-bit operands");
    static_assert(sizeof(TcCtrl) <= 1024, "control block");
    static_assert(!DUMP || RR > 0, "score dump needs uniform ranks");
    static_assert(RR == 0 || C::COLS % (RR ? RR : 1) == 0, "an epilogue warp owns whole components");
    pdl_enter();
    if (n_dev) n = *n_dev;                       // rows listed on the device
    // work unit: one CTA (128-row tiles) or one CTA pair (256-row tiles)
    constexpr int UM = PAIR ? 2 * TC_M : TC_M;
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    const int unit = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int nunits = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    const int mtiles = (n + UM - 1) / UM;
    if (unit >= mtiles) return;                  // whole CTA (pair) idle, before any setup
    const int ntiles_all = Rtot / BN;
    const int tile0 = DUMP ? (int)((long long)ntiles_all * blockIdx.y / gridDim.y) : 0;
    const int tile1 = DUMP ? (int)((long long)ntiles_all * (blockIdx.y + 1) / gridDim.y) : ntiles_all;
    if (tile1 <= tile0) return;
    const int ntiles = tile1 - tile0;
    const int my_m = (mtiles - unit + nunits - 1) / nunits;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = smem;                      // 2 x A_BYTES
    unsigned char *sB = smem + 2 * C::A_BYTES;
    TcCtrl *ctl = (TcCtrl *)(sB + C::STAGES * C::B_STAGE);
    float *mrg = (float *)((unsigned char *)ctl + 1024);  // [NG-1][128][MW] merge buffer of the column groups

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort_flag = &ctl->abort_flag;
    // pairs: waits on barriers that the other CTA (or its commits) arrive on
    // use cluster-scope acquire, and a timeout aborts both CTAs
#define TC_WAIT(bar, par) (PAIR ? mbar_wait_cluster((bar), (par), abort_flag) : mbar_wait((bar), (par), abort_flag))
    // an epilogue warp hands accumulator buffer b back to the MMA thread (of rank 0)
#define TC_FREE(b)                                                                  \
    do {                                                                            \
        if (PAIR && rank != 0u) mbar_arrive_cluster(mapa_rank(smem_u32(&ctl->t_empty[b]), 0u)); \
        else mbar_arrive(smem_u32(&ctl->t_empty[b]));                               \
    } while (0)

    if (threadIdx.x == 0) {
        ctl->abort_flag = 0;
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&ctl->a_full[i]), 1);
            mbar_init(smem_u32(&ctl->a_empty[i]), 1);
            mbar_init(smem_u32(&ctl->ap_full[i]), 1);
        }
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(smem_u32(&ctl->b_full[s]), 1);
            mbar_init(smem_u32(&ctl->b_empty[s]), 1);
            mbar_init(smem_u32(&ctl->bp_full[s]), 1);
        }
        for (int b = 0; b < C::NB; ++b) {
            mbar_init(smem_u32(&ctl->t_full[b]), 1);
            mbar_init(smem_u32(&ctl->t_empty[b]), PAIR ? 2 * C::EWS : C::EWS);  // one set reads a buffer
        }
        mbar_init(smem_u32(&ctl->drain), 1);
        mbar_init(smem_u32(&ctl->bye), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapB);
    }
    if (warp == 1) {
        // pairs: one warp of each CTA takes part in the pair's allocation (the
        // same columns in both)
        if constexpr (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                             smem_u32(&ctl->tmem_base))
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                             smem_u32(&ctl->tmem_base))
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    // pairs: both CTAs' barriers are initialised before either arrives remotely
    if constexpr (PAIR) cluster_sync_all();
    else __syncthreads();
    tc_fence_after();
    const uint32_t tbase = ctl->tmem_base;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            bool ok = true;
            for (int mt = 0; ok && mt < my_m; ++mt) {
                const int m0 = (unit + mt * nunits) * UM + (int)rank * TC_M;
                const int ab = mt & 1, around = mt >> 1;
                if (!TC_WAIT(smem_u32(&ctl->a_empty[ab]), (around & 1) ^ 1)) break;
                const uint32_t af = smem_u32(&ctl->a_full[ab]);
                unsigned char *dA = sA + ab * C::A_BYTES;
                mbar_expect_tx(af, C::A_BYTES);
                tma_load_2d(smem_u32(dA), &mapA, 0, m0, af);
                if (NT == 3) tma_load_2d(smem_u32(dA + C::A_TILE), &mapAlo, 0, m0, af);
                for (int it = 0; it < ntiles; ++it) {
                    const int gi = mt * ntiles + it;
                    const int s = gi % C::STAGES, round = gi / C::STAGES;
                    if (!TC_WAIT(smem_u32(&ctl->b_empty[s]), (round & 1) ^ 1)) {
                        ok = false;
                        break;
                    }
                    const uint32_t bf = smem_u32(&ctl->b_full[s]);
                    mbar_expect_tx(bf, C::B_STAGE);
                    unsigned char *dst = sB + s * C::B_STAGE;
                    const int brow = (tile0 + it) * BN + (int)rank * C::B_ROWS;
                    tma_load_2d(smem_u32(dst), &mapB, 0, brow, bf);
                    if (NT == 3) tma_load_2d(smem_u32(dst + C::B_TILE), &mapBlo, 0, brow, bf);
                }
            }
        }
    } else if (warp == 1 && PAIR && rank == 1) {
        // ------------------------------------------------ relay (pair rank 1)
        // forwards each of this CTA's operand tiles, once landed, to rank 0's
        // MMA thread (in the order that thread consumes them)
        if (lane == 0) {
            bool ok = true;
            for (int mt = 0; ok && mt < my_m; ++mt) {
                const int ab = mt & 1, around = mt >> 1;
                if (!TC_WAIT(smem_u32(&ctl->a_full[ab]), around & 1)) break;
                mbar_arrive_cluster(mapa_rank(smem_u32(&ctl->ap_full[ab]), 0u));
                for (int it = 0; it < ntiles; ++it) {
                    const int gi = mt * ntiles + it;
                    const int s = gi % C::STAGES, round = gi / C::STAGES;
                    if (!TC_WAIT(smem_u32(&ctl->b_full[s]), round & 1)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_cluster(mapa_rank(smem_u32(&ctl->bp_full[s]), 0u));
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            bool ok = true;
            for (int mt = 0; ok && mt < my_m; ++mt) {
                const int ab = mt & 1, around = mt >> 1;
                if (!TC_WAIT(smem_u32(&ctl->a_full[ab]), around & 1)) break;
                if (PAIR && !TC_WAIT(smem_u32(&ctl->ap_full[ab]), around & 1)) break;
                tc_fence_after();
                const uint32_t aHi = smem_u32(sA + ab * C::A_BYTES), aLo = aHi + C::A_TILE;
                for (int it = 0; it < ntiles; ++it) {
                    const int gi = mt * ntiles + it;
                    const int s = gi % C::STAGES, round = gi / C::STAGES;
                    const int b = gi % C::NB, tround = gi / C::NB;
                    if (!TC_WAIT(smem_u32(&ctl->b_full[s]), round & 1) ||
                        (PAIR && !TC_WAIT(smem_u32(&ctl->bp_full[s]), round & 1)) ||
                        !TC_WAIT(smem_u32(&ctl->t_empty[b]), (tround & 1) ^ 1)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tbase + (uint32_t)(b * BN);
                    const uint32_t bHi = smem_u32(sB + s * C::B_STAGE), bLo = bHi + C::B_TILE;
#pragma unroll
                    for (int k = 0; k < C::ROWB / 32; ++k) {  // reduction depth 64: 32-byte K steps
                        const uint32_t off = (uint32_t)(k * 32);
                        if constexpr (NT == 8) {
                            mma_f8(d, sdesc_sw64(aHi + off), sdesc_sw64(bHi + off), idesc, k > 0 ? 1u : 0u);
                        } else if constexpr (PAIR) {
                            mma_f16_pair(d, sdesc_sw128(aHi + off), sdesc_sw128(bHi + off), idesc, k > 0 ? 1u : 0u);
                            if (NT == 3) {
                                mma_f16_pair(d, sdesc_sw128(aLo + off), sdesc_sw128(bHi + off), idesc, 1u);
                                mma_f16_pair(d, sdesc_sw128(aHi + off), sdesc_sw128(bLo + off), idesc, 1u);
                            }
                        } else {
                            mma_f16(d, sdesc_sw128(aHi + off), sdesc_sw128(bHi + off), idesc, k > 0 ? 1u : 0u);
                            if (NT == 3) {
                                mma_f16(d, sdesc_sw128(aLo + off), sdesc_sw128(bHi + off), idesc, 1u);
                                mma_f16(d, sdesc_sw128(aHi + off), sdesc_sw128(bLo + off), idesc, 1u);
                            }
                        }
                    }
                    if constexpr (PAIR) {
                        mma_commit_pair(smem_u32(&ctl->b_empty[s]), 3);
                        mma_commit_pair(smem_u32(&ctl->t_full[b]), 3);
                    } else {
                        mma_commit(smem_u32(&ctl->b_empty[s]));
                        mma_commit(smem_u32(&ctl->t_full[b]));
                    }
                }
                // A buffer free once these MMAs complete
                if constexpr (PAIR) mma_commit_pair(smem_u32(&ctl->a_empty[ab]), 3);
                else mma_commit(smem_u32(&ctl->a_empty[ab]));
            }
            // drain: every MMA issued above has completed once this arrives
            if constexpr (PAIR) {
                // the pair's MMAs write the other CTA's tensor memory: wait for
                // them even after an abort, before the teardown handshake
                mma_commit_pair(smem_u32(&ctl->drain), 1);
                if (!mbar_wait_bounded(smem_u32(&ctl->drain), 0)) *abort_flag = 1;
            } else {
                mma_commit(smem_u32(&ctl->drain));
                mbar_wait(smem_u32(&ctl->drain), 0, abort_flag);
            }
        }
    } else {
        // ------------------------------------------------ epilogue (EW warps)
        const int q = warp & 3;                    // TMEM lane quarter this warp may access
        const int set = (warp - 2) / C::EWS;       // the set's tiles: those of its parity (two sets)
        const int h = ((warp - 2) % C::EWS) >> 2;  // column group of each accumulator tile
        const int part = set * C::NG + h;          // this warp's partial result of its rows
        const int row = 32 * q + lane;
        bool ok = true;
        for (int mt = 0; ok && mt < my_m; ++mt) {
            const int m0 = (unit + mt * nunits) * UM + (int)rank * TC_M;
            const int grow = m0 + row;
            const float zzr = grow < n ? zz[grow] : 0.0f;
            const float rs2 = (NT == 8 && grow < n) ? zsc2[grow] : 1.0f;  // 8-bit: row scale squared
            float s1 = FLT_MAX, s2 = FLT_MAX, acc = 0.0f;
            int k1 = 0, curk = -1;
            float cs[4] = {FLT_MAX, FLT_MAX, FLT_MAX, FLT_MAX};
            int ck[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
            for (int it = 0; it < ntiles; ++it) {
                const int gi = mt * ntiles + it;
                if (C::SETS > 1 && (gi & 1) != set) continue;  // buffer gi % NB belongs to the other set
                const int b = gi % C::NB, tround = gi / C::NB;
                // tcgen05.ld is warp-collective: every lane takes the same branch
                if (!__all_sync(0xffffffffu, TC_WAIT(smem_u32(&ctl->t_full[b]), tround & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // uniform ranks: each column group owns whole components of its
                // BN / NG columns; ragged ranks: one group takes the whole tile
                // (components may straddle any split of it).
                const int cbeg = RR ? h * C::COLS : 0;
                const int ncol = RR ? C::COLS : BN;
                const int col0 = (tile0 + it) * BN + cbeg;
                const uint32_t taddr = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + cbeg);
                if constexpr (RR > 0) {
                    // the warp's columns in one TMEM round trip; the buffer is
                    // handed back to the MMA warp before the arithmetic
                    uint32_t r[C::COLS];
                    tmem_ld_all<C::COLS>(taddr, r);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) TC_FREE(b);
#pragma unroll
                    for (int p = 0; p < C::COLS / RR; ++p) {
                        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
                        for (int j = 0; j < RR; j += 4) {
                            const float v0 = __uint_as_float(r[p * RR + j]), v1 = __uint_as_float(r[p * RR + j + 1]);
                            const float v2 = __uint_as_float(r[p * RR + j + 2]), v3 = __uint_as_float(r[p * RR + j + 3]);
                            sq_acc2(a0, a1, v0, v1);
                            sq_acc2(a2, a3, v2, v3);
                        }
                        float sq = (a0 + a1) + (a2 + a3);
                        const int k = col0 / RR + p;
                        if (NT == 8 && k < K) sq *= rs2 * __ldg(&tab.k8s2[k]);
                        if (k < K) {
                            const float sc = __ldg(&tab.cst_hi[k]) + __ldg(&tab.t_hi[k]) * zzr +
                                             (RR == 64 ? sq : -sq);
                            if (DUMP) {
                                if (grow < n) scores[(size_t)grow * K + k] = sc;
                            } else if (CAND) {
                                top4_inc(sc, k, cs, ck);
                            } else {
                                top2(sc, k, s1, s2, k1);
                            }
                        }
                    }
                } else {
                // ragged ranks: this warp's group of the tile, [g0, g1), whole
                // components of multiples of 8 columns; 8-column TMEM loads,
                // four in flight; one component lookup per 8 columns
                const int4 tg = __ldg(&tileg[tile0 + it]);
                const int gs[5] = {0, tg.y, tg.z, tg.w, BN};
                const int g0 = gs[h], g1 = gs[h + 1];
                const uint32_t tq = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN);
                const int tcol = (tile0 + it) * BN;
                for (int c = g0; c < g1; c += 32) {
                    uint32_t r[4][8];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (c + 8 * u < g1) tmem_ld8(tq + (uint32_t)(c + 8 * u), r[u]);
                    tmem_wait8x4(r);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (c + 8 * u >= g1) break;
                        const int k = __ldg(&colk[tcol + c + 8 * u]);
                        if (k != curk) {
                            if (curk >= 0) {
                                const float a8 = NT == 8 ? acc * rs2 * __ldg(&tab.k8s2[curk]) : acc;
                                const float sc = __ldg(&tab.cst_hi[curk]) + __ldg(&tab.t_hi[curk]) * zzr +
                                                 __ldg(&tab.sgn[curk]) * a8;
                                if (CAND) top4_inc(sc, curk, cs, ck);
                                else top2(sc, curk, s1, s2, k1);
                            }
                            curk = k;
                            acc = 0.0f;
                        }
                        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
                        sq_acc2(a0, a1, __uint_as_float(r[u][0]), __uint_as_float(r[u][1]));
                        sq_acc2(a2, a3, __uint_as_float(r[u][2]), __uint_as_float(r[u][3]));
                        sq_acc2(a0, a1, __uint_as_float(r[u][4]), __uint_as_float(r[u][5]));
                        sq_acc2(a2, a3, __uint_as_float(r[u][6]), __uint_as_float(r[u][7]));
                        acc += (a0 + a1) + (a2 + a3);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) TC_FREE(b);
                // the group ends with a whole component
                if (curk >= 0) {
                    const float a8 = NT == 8 ? acc * rs2 * __ldg(&tab.k8s2[curk]) : acc;
                    const float sc = __ldg(&tab.cst_hi[curk]) + __ldg(&tab.t_hi[curk]) * zzr +
                                     __ldg(&tab.sgn[curk]) * a8;
                    if (CAND) top4_inc(sc, curk, cs, ck);
                    else top2(sc, curk, s1, s2, k1);
                }
                curk = -1;
                acc = 0.0f;
                }
            }
            if (CAND) {
                // merge the parts' four best, then list the undecided patch
                if (C::NP > 1 && part > 0) {
                    float *m = mrg + ((part - 1) * TC_M + row) * 8;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        m[j] = cs[j];
                        m[4 + j] = __int_as_float(ck[j]);
                    }
                }
                if (C::NP > 1) asm volatile("bar.sync 1, %0;" ::"n"(32 * C::EW) : "memory");
                if (part == 0 && grow < n && ok) {
#pragma unroll
                    for (int o = 1; o < C::NP; ++o) {
                        const float *m = mrg + ((o - 1) * TC_M + row) * 8;
#pragma unroll
                        for (int j = 0; j < 4; ++j) top4(m[j], __float_as_int(m[4 + j]), cs, ck);
                    }
                    kstar[grow] = ck[0];
                    const float gp = cs[1] - cs[0];
                    gap[grow] = gp;
                    const float thr = tau_abs + tau_rel * zzr * __ldg(tab.tmax);
                    if (!(gp >= thr)) {
                        const float lim = cs[0] + thr;
                        const int f = atomicAdd(nflag, 1);
                        flag[f] = grow;
                        cand[f] = cs[3] < lim ? make_int4(-1, -1, -1, -1)
                                              : make_int4(ck[0], ck[1], cs[2] < lim ? ck[2] : -1, -1);
                    }
                }
                // mrg is reused; every warp leaves the tile loop together
                if (C::NP > 1) ok = bar_and(ok, 1, 32 * C::EW);
            } else if (!DUMP) {
                // merge the parts (their components interleave); among equal
                // scores the lowest component index wins
                if (C::NP > 1 && part > 0) {
                    float *m = mrg + ((part - 1) * TC_M + row) * 3;
                    m[0] = s1;
                    m[1] = s2;
                    m[2] = __int_as_float(k1);
                }
                if (C::NP > 1) asm volatile("bar.sync 1, %0;" ::"n"(32 * C::EW) : "memory");
                if (part == 0 && grow < n && ok) {
                    const int out = rowmap ? rowmap[grow] : grow;
                    float b1 = s1, b2 = s2;
                    int bk = k1;
#pragma unroll
                    for (int o = 1; o < C::NP; ++o) {
                        const float *m = mrg + ((o - 1) * TC_M + row) * 3;
                        const float t1 = m[0], t2 = m[1];
                        const int tk = __float_as_int(m[2]);
                        if (t1 < b1 || (t1 == b1 && tk < bk)) {
                            b2 = fminf(b1, t2); b1 = t1; bk = tk;
                        } else {
                            b2 = fminf(b2, t1);
                        }
                    }
                    kstar[out] = bk;
                    const float gp = b2 - b1;
                    gap[out] = gp;
                    const float thr = tau_abs + tau_rel * zzr * __ldg(tab.tmax);
                    if (!(gp >= thr)) flag[atomicAdd(nflag, 1)] = out;
                }
                // mrg is reused; every warp leaves the tile loop together
                if (C::NP > 1) ok = bar_and(ok, 1, 32 * C::EW);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) {
        // neither CTA frees its tensor memory or leaves while the other may
        // still reach into it: rank 0's MMAs have drained, and every remote
        // arrival of rank 1 precedes its side of this handshake
        if (threadIdx.x == 0) {
            mbar_arrive_cluster(mapa_rank(smem_u32(&ctl->bye), rank ^ 1u));
            // (longer than any wait of the other CTA, which ends within one
            // bound of its last progress)
            if (!mbar_wait_bounded(smem_u32(&ctl->bye), 0, 3)) ctl->abort_flag = 1;
        }
        __syncthreads();
    }
    if (warp == 1) {
        tc_fence_after();
        if constexpr (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
    }
    if (threadIdx.x == 0 && ctl->abort_flag) atomicExch(err, 1);
#undef TC_WAIT
#undef TC_FREE
}

template <int BN, int NT, int RR, bool DUMP = false, bool CAND = false>
static epll_status launch_tc(epll_gmm *g, const CUtensorMap &a, const CUtensorMap &alo,
                             const CUtensorMap &b, const CUtensorMap &blo, int n, const int *rowmap,
                             const int *n_dev, const float *zz, uint32_t idesc, float tau_abs,
                             float tau_rel, int *flag, int *nflag, cudaStream_t st,
                             float *scores = nullptr, int slices = 1, const float *zsc2 = nullptr)
{
    using Cfg = TcCfg<BN, NT, RR, CAND>;
    auto kern = k_proj_tc<BN, NT, RR, DUMP, CAND>;
    static bool attr = false;
    if (!attr) {
        EPLL_CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
        attr = true;
    }
    Workspace &ws = g->ws;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        EPLL_CU(cudaGetDevice(&dev));
        EPLL_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int mtiles = (n + TC_M - 1) / TC_M;
    int gx = slices > 1 ? (sms / slices > 0 ? sms / slices : 1) : sms;
    if (gx > mtiles) gx = mtiles;
    if (gx < 1) gx = 1;
    const dim3 grid(gx, slices);
    // the instrumentation covers the pass over every sampled patch only
    if (!n_dev) prof_begin(g, st);
    EPLL_CU(launch_pdl(kern, grid, dim3(Cfg::THREADS), Cfg::SMEM, st, a, alo, b, blo, n, rowmap, n_dev, g->K, g->Rtot, idesc, zz,
                                             g->d_colk, g->d_tileg, g->tab, tau_abs, tau_rel, ws.kstar, ws.gap, flag,
                                             nflag, cnt(g, CNT_ERR), scores, zsc2,
                                             reinterpret_cast<int4 *>(ws.cand)));
    if (!n_dev) prof_end(g, st, n);
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

// The first pass over n sampled patches (n known on the host) in clusters of
// two CTAs sharing each MMA (M = 256).  The basis maps have boxes of BN / 2
// rows (each CTA loads half of every basis tile); idesc is that of M = 128.
template <int BN, int NT, int RR, bool CAND>
static epll_status launch_tc_pair(epll_gmm *g, const CUtensorMap &a, const CUtensorMap &alo,
                                  const CUtensorMap &b, const CUtensorMap &blo, int n, const float *zz,
                                  uint32_t idesc, float tau_abs, float tau_rel, int *flag, int *nflag,
                                  cudaStream_t st)
{
    using Cfg = TcCfg<BN, NT, RR, CAND, true>;
    auto kern = k_proj_tc<BN, NT, RR, false, CAND, true>;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(Cfg::THREADS);
    cfg.dynamicSmemBytes = Cfg::SMEM;
    cfg.stream = st;
    cfg.attrs = at;
    static int clusters = -1;  // pairs resident at once
    if (clusters < 0) {
        EPLL_CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
        cfg.gridDim = dim3(2);
        cfg.numAttrs = 1;
        int nc = 0;
        EPLL_CU(cudaOccupancyMaxActiveClusters(&nc, kern, &cfg));
        if (nc < 1) {
            set_error("selection: a cluster of two CTAs cannot be resident (disable CTA pairs)");
            return EPLL_ECUDA;
        }
        clusters = nc;
    }
    const int mtiles = (n + 2 * TC_M - 1) / (2 * TC_M);
    int pairs = clusters < mtiles ? clusters : mtiles;
    if (pairs < 1) pairs = 1;
    cfg.gridDim = dim3(2 * pairs);
    cfg.numAttrs = t_pdl ? 2 : 1;
    const uint32_t idesc2 = (idesc & ~(0x1Fu << 24)) | ((uint32_t)(2 * TC_M >> 4) << 24);  // M = 256
    Workspace &ws = g->ws;
    prof_begin(g, st);
    EPLL_CU(cudaLaunchKernelEx(&cfg, kern, a, alo, b, blo, n, (const int *)nullptr, (const int *)nullptr, g->K,
                               g->Rtot, idesc2, zz, (const int *)g->d_colk, (const int4 *)g->d_tileg, g->tab,
                               tau_abs, tau_rel, ws.kstar, ws.gap, flag, nflag, cnt(g, CNT_ERR), (float *)nullptr,
                               (const float *)nullptr, reinterpret_cast<int4 *>(ws.cand)));
    prof_end(g, st, n);
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

template <int BN, int NT, bool CAND = false>
static epll_status dispatch_rr(epll_gmm *g, const CUtensorMap &a, const CUtensorMap &alo,
                               const CUtensorMap &b, const CUtensorMap &blo, int n, const int *rowmap,
                               const int *n_dev, const float *zz, uint32_t idesc, float tau_abs,
                               float tau_rel, int *flag, int *nflag, cudaStream_t st,
                               const float *zsc2 = nullptr, bool pair = false)
{
    if constexpr (BN == 256 && NT != 8) {
        if (pair) {
            if (rowmap || n_dev) return fail(EPLL_EINVAL, "selection: CTA pairs serve the first pass only");
#define EPLL_TCP_ARGS g, a, alo, b, blo, n, zz, idesc, tau_abs, tau_rel, flag, nflag, st
            switch (g->uniform_rank) {
            case 64: return launch_tc_pair<BN, NT, 64, CAND>(EPLL_TCP_ARGS);
            case 16: return launch_tc_pair<BN, NT, 16, CAND>(EPLL_TCP_ARGS);
            case 8: return launch_tc_pair<BN, NT, 8, CAND>(EPLL_TCP_ARGS);
            default: return launch_tc_pair<BN, NT, 0, CAND>(EPLL_TCP_ARGS);
            }
#undef EPLL_TCP_ARGS
        }
    }
#define EPLL_TC_ARGS g, a, alo, b, blo, n, rowmap, n_dev, zz, idesc, tau_abs, tau_rel, flag, nflag, st, nullptr, 1, zsc2
    switch (g->uniform_rank) {
    case 64: return launch_tc<BN, NT, 64, false, CAND>(EPLL_TC_ARGS);
    case 16: return launch_tc<BN, NT, 16, false, CAND>(EPLL_TC_ARGS);
    case 8: return launch_tc<BN, NT, 8, false, CAND>(EPLL_TC_ARGS);
    default: return launch_tc<BN, NT, 0, false, CAND>(EPLL_TC_ARGS);
    }
#undef EPLL_TC_ARGS
}

// Split-BF16 scores of every component for the rows of the near-tie list
// (ws.flag, device count): the candidates of the compensated rescoring are the
// components within the split form's error band of the best.  Returns
// EPLL_EUNSUPPORTED for ragged ranks (the FP32 list-mode kernel serves them).
epll_status launch_dump_split(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                              cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int RR = g->uniform_rank;
    if (RR == 0 || (size_t)n > ws.fcap) return EPLL_EUNSUPPORTED;
    const int rows = (n + TC_M - 1) / TC_M * TC_M;
    uint16_t *Z2hi = ws.Z2, *Z2lo = ws.Z2 + ws.zrows * PD;
    int *nf = cnt(g, CNT_NFLAG);
    epll_status s;
    if ((s = launch_extract(g, xhat, H, W, anchors, n, ws.flag, nf, 1, 1, Z2hi, Z2lo, ws.zz2, nullptr, nullptr, st)))
        return s;
    CUtensorMap a2, a2lo, bs, bslo;
    if ((s = make_map(&a2, Z2hi, rows, TC_M))) return s;
    if ((s = make_map(&a2lo, Z2lo, rows, TC_M))) return s;
    if ((s = make_map(&bs, g->tab.Bs, g->Rtot, 128))) return s;
    if ((s = make_map(&bslo, g->tab.Bs_lo, g->Rtot, 128))) return s;
    const int ntiles = g->Rtot / 128;
    const int slices = ntiles < 32 ? ntiles : 32;
    const uint32_t idesc = idesc_f16(TC_M, 128, 1);
#define EPLL_DUMP_ARGS g, a2, a2lo, bs, bslo, n, ws.flag, nf, ws.zz2, idesc, 0.0f, 0.0f, nullptr, nullptr, st, ws.fscore, slices, nullptr
    switch (RR) {
    case 64: return launch_tc<128, 3, 64, true>(EPLL_DUMP_ARGS);
    case 16: return launch_tc<128, 3, 16, true>(EPLL_DUMP_ARGS);
    default: return launch_tc<128, 3, 8, true>(EPLL_DUMP_ARGS);
    }
#undef EPLL_DUMP_ARGS
}

// Gaussian selection on the tensor cores.
// BF16X3: the split pass scores every sampled patch; its near-ties go to the
// compensated FP32 rescoring (ws.flag).
// FP16: a one-term pass scores every sampled patch and keeps each patch's
// four best components; a patch it cannot decide is listed with the
// components within its error bound of the best, and these (patch,
// component) pairs are grouped by component and rescored in the split form
// (launch_pair_scores); what that cannot decide, and every patch whose band
// may hold more than four components, goes to the compensated rescoring.
// The split rows and means of every patch are extracted beside the FP16
// operand, for the estimation step.
// BF16 / FP8: a one-term pass; the rows it cannot decide (a third or more of
// them for BF16) are rescored by the split pass over every component, whose
// near-ties go to the compensated rescoring.
epll_status launch_select_tc(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                             int precision, float tau_abs, float tau_rel, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const bool split_first = precision == EPLL_BF16X3;
    const bool fp8 = precision == EPLL_FP8;
    const int fmt = precision == EPLL_FP16 ? 2 : (fp8 ? 3 : 1);
    const int rows = (n + TC_M - 1) / TC_M * TC_M;
    uint16_t *Zhi = ws.Zb, *Zlo = ws.Zb + ws.zrows * PD;
    epll_status s;
    // the ragged-rank layout is packed in 256-column tiles
    const bool bn128 = g->tile_bn == 128 && g->uniform_rank != 0;
    const int BNs = bn128 ? 128 : 256;
    // CTA pairs (first pass, 256-column tiles, 16-bit operands): each CTA of
    // a pair loads half of every basis tile
    const bool pair = g->tc_pair && !bn128 && !fp8;
    const int bbox = pair ? BNs / 2 : BNs;
    if (fmt == 2) {
        if ((s = ensure_prop_ws(g, n))) return s;  // ws.cand, the pair buffers
        // FP16 operand rows in ws.Z2 (free until the rescoring's score dump)
        uint16_t *Zf = ws.Z2;
        if ((s = launch_extract(g, xhat, H, W, anchors, n, nullptr, nullptr, 1, 1, Zhi, Zlo, ws.zz, nullptr, ws.mu,
                                st, Zf)))
            return s;
        int *nflag1 = cnt(g, CNT_NFLAG1);
        EPLL_CU(cudaMemsetAsync(nflag1, 0, sizeof(int), st));
        EPLL_CU(cudaMemsetAsync(cnt(g, CNT_NFLAG), 0, sizeof(int), st));
        CUtensorMap a, b;
        if ((s = make_map(&a, Zf, rows, TC_M))) return s;
        if ((s = make_map(&b, g->tab.B1, g->Rtot, bbox))) return s;
        if ((s = bn128 ? dispatch_rr<128, 1, true>(g, a, a, b, b, n, nullptr, nullptr, ws.zz, idesc_f16(TC_M, 128, 0),
                                                   tau_abs, tau_rel, ws.flag1, nflag1, st)
                       : dispatch_rr<256, 1, true>(g, a, a, b, b, n, nullptr, nullptr, ws.zz, idesc_f16(TC_M, 256, 0),
                                                   tau_abs, tau_rel, ws.flag1, nflag1, st, nullptr, pair)))
            return s;
        if ((s = launch_pair_scores(g, xhat, H, W, anchors, n, 4, ws.flag1, nflag1, st))) return s;
        return launch_cand_combine(g, n, 4, ws.flag1, nflag1, tau_abs, ws.flag, cnt(g, CNT_NFLAG), st);
    }
    // ---- first pass over every sampled patch
    if ((s = launch_extract(g, xhat, H, W, anchors, n, nullptr, nullptr, fmt, split_first ? 1 : 0, Zhi, Zlo, ws.zz,
                            ws.zsc2, split_first ? ws.mu : nullptr, st)))
        return s;
    int *flag1 = split_first ? ws.flag : ws.flag1;
    int *nflag1 = cnt(g, split_first ? CNT_NFLAG : CNT_NFLAG1);
    EPLL_CU(cudaMemsetAsync(nflag1, 0, sizeof(int), st));
    CUtensorMap a, alo, b, blo;
    if ((s = make_map(&a, Zhi, rows, TC_M))) return s;
    if ((s = make_map(&alo, Zlo, rows, TC_M))) return s;
    if (split_first) {
        if ((s = make_map(&b, g->tab.Bs, g->Rtot, bbox))) return s;
        if ((s = make_map(&blo, g->tab.Bs_lo, g->Rtot, bbox))) return s;
        return bn128 ? dispatch_rr<128, 3>(g, a, alo, b, blo, n, nullptr, nullptr, ws.zz, idesc_f16(TC_M, 128, 1),
                                           tau_abs, tau_rel, flag1, nflag1, st)
                     : dispatch_rr<256, 3>(g, a, alo, b, blo, n, nullptr, nullptr, ws.zz, idesc_f16(TC_M, 256, 1),
                                           tau_abs, tau_rel, flag1, nflag1, st, nullptr, pair);
    }
    if (fp8) {
        CUtensorMap a8, b8;
        if ((s = make_map(&a8, Zhi, rows, TC_M, 1))) return s;
        if ((s = make_map(&b8, g->tab.B8, g->Rtot, 256, 1))) return s;
        // one E4M3 product (kind::f8f6f4, E4M3 = format 0); scales folded into the epilogue
        if ((s = dispatch_rr<256, 8>(g, a8, a8, b8, b8, n, nullptr, nullptr, ws.zz, idesc_f16(TC_M, 256, 0),
                                     tau_abs, tau_rel, flag1, nflag1, st, ws.zsc2)))
            return s;
    } else {
        if ((s = make_map(&b, g->tab.B1, g->Rtot, pair ? 128 : 256))) return s;
        // one-term BF16 pass: no lo operands (the lo map arguments are unused)
        if ((s = dispatch_rr<256, 1>(g, a, a, b, b, n, nullptr, nullptr, ws.zz, idesc_f16(TC_M, 256, 1), tau_abs,
                                     tau_rel, flag1, nflag1, st, nullptr, pair)))
            return s;
    }
    return launch_split_pass(g, xhat, H, W, anchors, n, flag1, nflag1, tau_abs, st);
}

// Split-BF16 pass over the rows listed in flag1 (device count nflag1): their
// kstar / gap are overwritten and the rows it cannot decide go to ws.flag.
epll_status launch_split_pass(epll_gmm *g, const float *xhat, int H, int W, const int *anchors, int n,
                              const int *flag1, const int *nflag1, float tau_abs, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int rows = (n + TC_M - 1) / TC_M * TC_M;
    epll_status s;
    uint16_t *Z2hi = ws.Z2, *Z2lo = ws.Z2 + ws.zrows * PD;
    if ((s = launch_extract(g, xhat, H, W, anchors, n, flag1, nflag1, 1, 1, Z2hi, Z2lo, ws.zz2, nullptr, nullptr,
                            st)))
        return s;
    EPLL_CU(cudaMemsetAsync(cnt(g, CNT_NFLAG), 0, sizeof(int), st));
    CUtensorMap a2, a2lo, bs, bslo;
    if ((s = make_map(&a2, Z2hi, rows, TC_M))) return s;
    if ((s = make_map(&a2lo, Z2lo, rows, TC_M))) return s;
    const bool bn128 = g->tile_bn == 128 && g->uniform_rank != 0;
    if ((s = make_map(&bs, g->tab.Bs, g->Rtot, bn128 ? 128 : 256))) return s;
    if ((s = make_map(&bslo, g->tab.Bs_lo, g->Rtot, bn128 ? 128 : 256))) return s;
    return bn128 ? dispatch_rr<128, 3>(g, a2, a2lo, bs, bslo, n, flag1, nflag1, ws.zz2, idesc_f16(TC_M, 128, 1),
                                       tau_abs, SPLIT_REL, ws.flag, cnt(g, CNT_NFLAG), st)
                 : dispatch_rr<256, 3>(g, a2, a2lo, bs, bslo, n, flag1, nflag1, ws.zz2, idesc_f16(TC_M, 256, 1),
                                       tau_abs, SPLIT_REL, ws.flag, cnt(g, CNT_NFLAG), st);
}

}  // namespace epll
