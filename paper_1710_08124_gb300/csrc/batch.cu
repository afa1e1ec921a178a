// Batched restoration of images of uneven size, noise level and degradation.
//
// Small images leave most of the GPU idle (a 128 x 128 image at a 1/3 subset
// is 43 row tiles of the selection kernel for 152 SMs), so the batch is spread
// over lanes: contexts that share the handle's model arrays and own their
// tables (the per-beta tables are per image) and workspace, each on its own
// stream.  Images are assigned largest first to the least-loaded lane.  The
// whole batch -- every lane's HQS iterations, forked from and joined back to
// one origin stream -- is captured once into a CUDA graph; later calls with
// the same job list replay it with a single launch.  With lanes = 0 the lane
// count is tuned on the first call by timing the graph for 1, 2, 4 and 8
// lanes, then the tile shapes (selection basis columns per stage,
// reprojection threads per pixel group) at that lane count.  Periodic-blur
// jobs read their kernels from a device copy made at every call.
#include "epll_internal.cuh"

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

namespace epll {

constexpr int MAX_LANES = 8;

struct BatchState {
    std::vector<epll_gmm *> lanes;
    std::vector<cudaStream_t> streams;
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;        // what the captured graph runs
    std::vector<unsigned char> tuned_key;  // job list the tuned configuration belongs to
    int tuned_lanes = 0, tuned_bn = 256, tuned_agg = 1;
    float *d_kern = nullptr;               // device copies of the jobs' blur kernels
    size_t kern_cap = 0;
    std::vector<size_t> kern_off;          // per job: offset in d_kern (CONV jobs)
};

// One tile configuration of the autotuner.
struct TileCfg {
    int bn, agg;
};

epll_gmm *make_lane(const epll_gmm *g)
{
    epll_gmm *l = new epll_gmm();
    l->K = g->K;
    l->Rtot = g->Rtot;
    l->uniform_rank = g->uniform_rank;
    l->rank_mode = g->rank_mode;
    l->rank_param = g->rank_param;
    l->h_r = g->h_r;
    l->h_lam = g->h_lam;
    l->h_roff = g->h_roff;
    l->d_r = g->d_r;
    l->d_roff = g->d_roff;
    l->d_colk = g->d_colk;
    l->d_tileg = g->d_tileg;
    l->d_S = g->d_S;
    l->d_w = g->d_w;
    l->d_lam = g->d_lam;
    l->d_B = g->d_B;
    l->d_Blo = g->d_Blo;
    l->d_Ub = g->d_Ub;
    l->d_U2b = g->d_U2b;
    l->Rp = g->Rp;
    l->rank_sum = g->rank_sum;
    l->lane = true;
    if (alloc_tables(l) != cudaSuccess) {
        cudaGetLastError();
        epll_gmm_free(l);
        return nullptr;
    }
    return l;
}

void free_batch(epll_gmm *g)
{
    BatchState *b = g->batch;
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (epll_gmm *l : b->lanes) epll_gmm_free(l);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->t0) cudaEventDestroy(b->t0);
    if (b->t1) cudaEventDestroy(b->t1);
    if (b->d_kern) cudaFree(b->d_kern);
    delete b;
    g->batch = nullptr;
}

template <typename T>
static void put(std::vector<unsigned char> &k, const T &v)
{
    const unsigned char *p = reinterpret_cast<const unsigned char *>(&v);
    k.insert(k.end(), p, p + sizeof(T));
}

static std::vector<unsigned char> job_key(const epll_gmm *g, int n, const epll_job *jobs, const double *beta,
                                          int T, const epll_options &o)
{
    std::vector<unsigned char> k;
    put(k, g->prop);
    put(k, g->tree);
    put(k, g->prop_topm);
    put(k, g->prop_pmin);
    put(k, n);
    for (int i = 0; i < n; ++i) put(k, jobs[i]);
    put(k, T);
    for (int t = 0; t < T; ++t) put(k, beta[t]);
    put(k, o);
    return k;
}

// Largest image first onto the lane with the fewest pixels so far.
static std::vector<std::vector<int>> assign(int n, const epll_job *jobs, int L)
{
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)jobs[a].H * jobs[a].W > (long long)jobs[b].H * jobs[b].W;
    });
    std::vector<std::vector<int>> lanes(L);
    std::vector<long long> load(L, 0);
    for (int j : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lanes[l].push_back(j);
        load[l] += (long long)jobs[j].H * jobs[j].W;
    }
    return lanes;
}

// dkern: the job's blur kernel in device memory (CONV jobs in a graph), or
// nullptr to use the host kernel of the job.
static epll_status run_job(epll_gmm *ctx, const epll_job &j, const double *beta, int T,
                           const epll_options &o, cudaStream_t st, const float *dkern = nullptr)
{
    const bool conv = j.kind == EPLL_CONV_PERIODIC;
    epll_degradation deg{j.kind, j.a, conv ? (dkern ? dkern : j.kernel) : nullptr, conv ? j.kh : 0,
                         conv ? j.kw : 0, 1};
    epll_status s = run_restore(ctx, j.y, j.kind == EPLL_PIXELWISE ? j.a : nullptr, j.H, j.W, &deg, j.sigma,
                                beta, T, o, st, conv && dkern != nullptr);
    if (s) return s;
    EPLL_CU(cudaMemcpyAsync(j.x_out, ctx->ws.xhat, sizeof(float) * (size_t)j.H * j.W,
                            cudaMemcpyDeviceToDevice, st));
    return EPLL_OK;
}

// Lanes, streams, events and workspaces for L lanes (allocation happens here,
// never while a graph is being captured).
static epll_status prepare_lanes(epll_gmm *g, BatchState *b, const std::vector<std::vector<int>> &part,
                                 const epll_job *jobs)
{
    const int L = (int)part.size();
    if (!b->origin) EPLL_CU(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking));
    if (!b->fork) EPLL_CU(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    if (!b->t0) EPLL_CU(cudaEventCreate(&b->t0));
    if (!b->t1) EPLL_CU(cudaEventCreate(&b->t1));
    while ((int)b->lanes.size() < L) {
        epll_gmm *l = make_lane(g);
        if (!l) return fail(EPLL_ENOMEM, "batch lane allocation failed");
        b->lanes.push_back(l);
        cudaStream_t s;
        cudaEvent_t e;
        EPLL_CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        EPLL_CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->streams.push_back(s);
        b->join.push_back(e);
    }
    for (int l = 0; l < L; ++l) {
        size_t maxN = 0;
        for (int j : part[l]) maxN = std::max(maxN, (size_t)jobs[j].H * jobs[j].W);
        epll_status s;
        if ((s = ensure_workspace(b->lanes[l], maxN))) return s;
        b->lanes[l]->prop = g->prop;
        b->lanes[l]->prop_topm = g->prop_topm;
        b->lanes[l]->prop_pmin = g->prop_pmin;
        b->lanes[l]->tc_pair = g->tc_pair;
        // the tree: a lane of the node model (own tables), the handle's arrays
        epll_gmm *ln = b->lanes[l];
        if (!(ln->tree && ln->tree->src == g->tree)) {
            free_tree(ln);
            if (g->tree) {
                TreeState *tr = new TreeState(*g->tree);
                tr->owns_arrays = false;
                tr->src = g->tree;
                tr->tm = make_lane(g->tree->tm);
                if (!tr->tm) {
                    delete tr;
                    return fail(EPLL_ENOMEM, "batch lane tree allocation failed");
                }
                ln->tree = tr;
            }
        }
    }
    return EPLL_OK;
}

// Forks the lanes from `origin`, issues every lane's images, joins them back.
static epll_status issue(BatchState *b, const std::vector<std::vector<int>> &part, const epll_job *jobs,
                         const double *beta, int T, const epll_options &o, cudaStream_t origin)
{
    // lanes run side by side: no programmatic early launch (see t_pdl)
    struct PdlOff {
        PdlOff() { t_pdl = false; }
        ~PdlOff() { t_pdl = true; }
    } pdl_off;
    EPLL_CU(cudaEventRecord(b->fork, origin));
    for (size_t l = 0; l < part.size(); ++l) {
        EPLL_CU(cudaStreamWaitEvent(b->streams[l], b->fork, 0));
        for (int j : part[l]) {
            const float *dk = jobs[j].kind == EPLL_CONV_PERIODIC ? b->d_kern + b->kern_off[j] : nullptr;
            epll_status s = run_job(b->lanes[l], jobs[j], beta, T, o, b->streams[l], dk);
            if (s) return s;
        }
        EPLL_CU(cudaEventRecord(b->join[l], b->streams[l]));
        EPLL_CU(cudaStreamWaitEvent(origin, b->join[l], 0));
    }
    return EPLL_OK;
}

// Eager run (lazy initialisations happen here), then capture and instantiate.
static epll_status build_graph(epll_gmm *g, BatchState *b, int n, const epll_job *jobs, const double *beta,
                               int T, const epll_options &o, int L, TileCfg tc, cudaStream_t st)
{
    const auto part = assign(n, jobs, L);
    epll_status s;
    if ((s = prepare_lanes(g, b, part, jobs))) return s;
    for (int l = 0; l < L; ++l) {
        b->lanes[l]->tile_bn = tc.bn;
        b->lanes[l]->tile_agg = tc.agg;
    }
    if ((s = issue(b, part, jobs, beta, T, o, st))) return s;
    EPLL_CU(cudaStreamSynchronize(st));
    if (b->exec) {
        EPLL_CU(cudaGraphExecDestroy(b->exec));
        b->exec = nullptr;
    }
    b->key.clear();
    EPLL_CU(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
    s = issue(b, part, jobs, beta, T, o, b->origin);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->origin, &graph);
    if (s) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return fail(EPLL_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return fail(EPLL_ECUDA, std::string("graph instantiation: ") + cudaGetErrorString(e));
    }
    return EPLL_OK;
}

}  // namespace epll

using namespace epll;

extern "C" epll_status epll_restore_batch(epll_gmm *g, int n, const epll_job *jobs, const double *beta_mult,
                                          int T, const epll_options *opt, int mode, int lanes, void *stream)
{
    if (!g || g->lane) return fail(EPLL_EINVAL, "null model handle");
    if (n < 1 || !jobs) return fail(EPLL_EINVAL, "batch needs at least one job");
    if (mode != EPLL_BATCH_SEQUENTIAL && mode != EPLL_BATCH_GRAPH) return fail(EPLL_EINVAL, "unknown batch mode");
    if (lanes < 0 || lanes > MAX_LANES) return fail(EPLL_EINVAL, "lanes must be in 0..8");
    epll_options o;
    if (opt) o = *opt; else epll_options_default(&o);
    size_t maxN = 0, kern_total = 0;
    for (int i = 0; i < n; ++i) {
        const epll_job &j = jobs[i];
        if (j.kind != EPLL_DENOISE && j.kind != EPLL_PIXELWISE && j.kind != EPLL_CONV_PERIODIC)
            return fail(EPLL_EINVAL, "batch jobs are EPLL_DENOISE, EPLL_PIXELWISE or EPLL_CONV_PERIODIC");
        const bool conv = j.kind == EPLL_CONV_PERIODIC;
        epll_degradation deg{j.kind, j.a, conv ? j.kernel : nullptr, conv ? j.kh : 0, conv ? j.kw : 0, 1};
        epll_status s = check_restore_args(g, j.y, j.H, j.W, &deg, j.sigma, beta_mult, T, o, j.x_out);
        if (s) return s;
        maxN = std::max(maxN, (size_t)j.H * j.W);
        if (conv) kern_total += (size_t)j.kh * j.kw;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (mode == EPLL_BATCH_SEQUENTIAL) {
        epll_status s;
        if ((s = ensure_workspace(g, maxN))) return s;
        for (int i = 0; i < n; ++i)
            if ((s = run_job(g, jobs[i], beta_mult, T, o, st))) return s;
        return EPLL_OK;
    }
    if (!g->batch) g->batch = new BatchState();
    BatchState *b = g->batch;
    // device copies of the blur kernels (before any capture; refreshed at every call)
    b->kern_off.assign((size_t)n, 0);
    if (kern_total) {
        if (kern_total > b->kern_cap) {
            EPLL_CU(cudaDeviceSynchronize());
            if (b->d_kern) cudaFree(b->d_kern);
            b->d_kern = nullptr;
            b->kern_cap = 0;
            EPLL_CU(cudaMalloc(&b->d_kern, sizeof(float) * kern_total));
            b->kern_cap = kern_total;
        }
        std::vector<float> hk(kern_total);
        size_t off = 0;
        for (int i = 0; i < n; ++i)
            if (jobs[i].kind == EPLL_CONV_PERIODIC) {
                b->kern_off[i] = off;
                std::memcpy(hk.data() + off, jobs[i].kernel, sizeof(float) * (size_t)jobs[i].kh * jobs[i].kw);
                off += (size_t)jobs[i].kh * jobs[i].kw;
            }
        EPLL_CU(cudaMemcpyAsync(b->d_kern, hk.data(), sizeof(float) * kern_total, cudaMemcpyHostToDevice, st));
        EPLL_CU(cudaStreamSynchronize(st));
    }
    const std::vector<unsigned char> jk = job_key(g, n, jobs, beta_mult, T, o);
    int L = lanes;
    TileCfg tc{g->tile_bn, g->tile_agg};
    if (L == 0) {
        if (b->tuned_key == jk && b->tuned_lanes > 0) {
            L = b->tuned_lanes;
            tc = TileCfg{b->tuned_bn, b->tuned_agg};
        } else {
            // time a captured configuration (one warm replay, then two timed)
            auto time_cfg = [&](int cand, TileCfg c, float *ms) -> epll_status {
                epll_status s = build_graph(g, b, n, jobs, beta_mult, T, o, cand, c, st);
                if (s) return s;
                b->key.clear();  // the tuning graphs are not reused
                EPLL_CU(cudaGraphLaunch(b->exec, st));
                EPLL_CU(cudaEventRecord(b->t0, st));
                EPLL_CU(cudaGraphLaunch(b->exec, st));
                EPLL_CU(cudaGraphLaunch(b->exec, st));
                EPLL_CU(cudaEventRecord(b->t1, st));
                EPLL_CU(cudaEventSynchronize(b->t1));
                EPLL_CU(cudaEventElapsedTime(ms, b->t0, b->t1));
                return EPLL_OK;
            };
            // lanes 1, 2, 4, 8 with the handle's tiles, then the tile shapes
            float best = 0.0f;
            int bestL = 1;
            for (int cand = 1; cand <= MAX_LANES && cand <= n; cand *= 2) {
                float ms = 0.0f;
                epll_status s = time_cfg(cand, tc, &ms);
                if (s) return s;
                if (cand == 1 || ms < best) {
                    best = ms;
                    bestL = cand;
                }
            }
            TileCfg bestT = tc;
            const TileCfg alts[] = {{128, tc.agg}, {tc.bn, tc.agg == 2 ? 1 : 2}};
            for (const TileCfg &c : alts) {
                if (c.bn == tc.bn && c.agg == tc.agg) continue;
                float ms = 0.0f;
                epll_status s = time_cfg(bestL, c, &ms);
                if (s) return s;
                if (ms < best) {
                    best = ms;
                    bestT = c;
                }
            }
            b->tuned_key = jk;
            b->tuned_lanes = bestL;
            b->tuned_bn = bestT.bn;
            b->tuned_agg = bestT.agg;
            L = bestL;
            tc = bestT;
        }
    }
    L = std::min(L, n);
    std::vector<unsigned char> key = jk;
    put(key, L);
    put(key, tc.bn);
    put(key, tc.agg);
    put(key, g->tc_pair);
    if (!(b->exec && b->key == key)) {
        epll_status s = build_graph(g, b, n, jobs, beta_mult, T, o, L, tc, st);
        if (s) return s;
        b->key = key;
    }
    EPLL_CU(cudaGraphLaunch(b->exec, st));
    return EPLL_OK;
}

extern "C" epll_status epll_set_tiles(epll_gmm *g, int tile_bn, int tile_agg)
{
    if (!g || g->lane) return fail(EPLL_EINVAL, "null model handle");
    if ((tile_bn != 128 && tile_bn != 256) || (tile_agg != 1 && tile_agg != 2))
        return fail(EPLL_EINVAL, "tile_bn must be 128 or 256 and tile_agg 1 or 2");
    g->tile_bn = tile_bn;
    g->tile_agg = tile_agg;
    return EPLL_OK;
}

extern "C" epll_status epll_set_cta_pairs(epll_gmm *g, int enable)
{
    if (!g || g->lane) return fail(EPLL_EINVAL, "null model handle");
    if (enable != 0 && enable != 1) return fail(EPLL_EINVAL, "enable must be 0 or 1");
    g->tc_pair = enable;
    return EPLL_OK;
}

extern "C" epll_status epll_batch_config(epll_gmm *g, int *lanes, int *tile_bn, int *tile_agg)
{
    if (!g || g->lane) return fail(EPLL_EINVAL, "null model handle");
    const BatchState *b = g->batch;
    if (lanes) *lanes = b ? b->tuned_lanes : 0;
    if (tile_bn) *tile_bn = b && b->tuned_lanes ? b->tuned_bn : g->tile_bn;
    if (tile_agg) *tile_agg = b && b->tuned_lanes ? b->tuned_agg : g->tile_agg;
    return EPLL_OK;
}
