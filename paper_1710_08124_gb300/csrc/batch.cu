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
// lanes.
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
    std::vector<unsigned char> tuned_key;  // job list the tuned lane count belongs to
    int tuned_lanes = 0;
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

static epll_status run_job(epll_gmm *ctx, const epll_job &j, const double *beta, int T,
                           const epll_options &o, cudaStream_t st)
{
    epll_degradation deg{j.kind, j.a, nullptr, 0, 0, 1};
    epll_status s = run_restore(ctx, j.y, j.kind == EPLL_PIXELWISE ? j.a : nullptr, j.H, j.W, &deg, j.sigma,
                                beta, T, o, st);
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
    EPLL_CU(cudaEventRecord(b->fork, origin));
    for (size_t l = 0; l < part.size(); ++l) {
        EPLL_CU(cudaStreamWaitEvent(b->streams[l], b->fork, 0));
        for (int j : part[l]) {
            epll_status s = run_job(b->lanes[l], jobs[j], beta, T, o, b->streams[l]);
            if (s) return s;
        }
        EPLL_CU(cudaEventRecord(b->join[l], b->streams[l]));
        EPLL_CU(cudaStreamWaitEvent(origin, b->join[l], 0));
    }
    return EPLL_OK;
}

// Eager run (lazy initialisations happen here), then capture and instantiate.
static epll_status build_graph(epll_gmm *g, BatchState *b, int n, const epll_job *jobs, const double *beta,
                               int T, const epll_options &o, int L, cudaStream_t st)
{
    const auto part = assign(n, jobs, L);
    epll_status s;
    if ((s = prepare_lanes(g, b, part, jobs))) return s;
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
    size_t maxN = 0;
    for (int i = 0; i < n; ++i) {
        const epll_job &j = jobs[i];
        if (j.kind != EPLL_DENOISE && j.kind != EPLL_PIXELWISE)
            return fail(EPLL_EINVAL, "batch jobs are EPLL_DENOISE or EPLL_PIXELWISE");
        epll_degradation deg{j.kind, j.a, nullptr, 0, 0, 1};
        epll_status s = check_restore_args(g, j.y, j.H, j.W, &deg, j.sigma, beta_mult, T, o, j.x_out);
        if (s) return s;
        maxN = std::max(maxN, (size_t)j.H * j.W);
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
    const std::vector<unsigned char> jk = job_key(g, n, jobs, beta_mult, T, o);
    int L = lanes;
    if (L == 0) {
        if (b->tuned_key == jk && b->tuned_lanes > 0) {
            L = b->tuned_lanes;
        } else {
            // time the captured batch for 1, 2, 4, 8 lanes (two replays each)
            float best = 0.0f;
            int bestL = 1;
            for (int cand = 1; cand <= MAX_LANES && cand <= n; cand *= 2) {
                epll_status s = build_graph(g, b, n, jobs, beta_mult, T, o, cand, st);
                if (s) return s;
                EPLL_CU(cudaGraphLaunch(b->exec, st));
                EPLL_CU(cudaEventRecord(b->t0, st));
                EPLL_CU(cudaGraphLaunch(b->exec, st));
                EPLL_CU(cudaGraphLaunch(b->exec, st));
                EPLL_CU(cudaEventRecord(b->t1, st));
                EPLL_CU(cudaEventSynchronize(b->t1));
                float ms = 0.0f;
                EPLL_CU(cudaEventElapsedTime(&ms, b->t0, b->t1));
                if (cand == 1 || ms < best) {
                    best = ms;
                    bestL = cand;
                }
                b->key = jk;
                put(b->key, cand);
            }
            b->tuned_key = jk;
            b->tuned_lanes = bestL;
            L = bestL;
        }
    }
    L = std::min(L, n);
    std::vector<unsigned char> key = jk;
    put(key, L);
    if (!(b->exec && b->key == key)) {
        epll_status s = build_graph(g, b, n, jobs, beta_mult, T, o, L, st);
        if (s) return s;
        b->key = key;
    }
    EPLL_CU(cudaGraphLaunch(b->exec, st));
    return EPLL_OK;
}
