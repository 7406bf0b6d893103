// sf_api.cu -- the C-ABI of the vehicle step (include/sf.h).
//
// Host side: argument validation, the derived road store built once at load
// time, device allocations, the exchange layout of the agent state,
// checkpoints and the device error word; and the episode-metrics pass (a
// small kernel after each step).  Every step computation runs in the kernels
// of sf_world.cu.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <utility>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sf.h"
#include "sf_internal.cuh"
#include "sf_mlp_internal.cuh"

namespace {

thread_local std::string g_create_error;

// counters of the episode metrics, in the order of sf_metrics
enum : int {
    kMetricEpisodes = 0, kMetricGoals, kMetricCollisions, kMetricCrashes, kMetricOffroad, kMetricLaneForb,
    kMetricIdle, kMetricTimeouts, kMetricNonfinite, kMetricDracOver, kMetricDracMicro, kMetricCount
};

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
};

}  // namespace

struct sf_ctx {
    sf_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    int W = 0, A = 0, NP = 0;
    std::vector<void*> allocs;
    DevState st{};
    DevRoads rd{};
    DevOutputs out{};
    float* place_buf = nullptr;
    uint8_t* all_mask = nullptr;
    float* act_buf = nullptr;   // [A][3] actions written by an attached policy
    // episode metrics (SF_FLAG_METRICS): per agent the running episode's maximum DRAC
    // and event bits; the counters of the ended episodes (kMetric*)
    float* m_epmax = nullptr;
    uint32_t* m_epev = nullptr;
    unsigned long long* m_cnt = nullptr;
    void* surr = nullptr;       // surrogate step buffers (allocated on first use)
    void* lfb = nullptr;        // full observation and critic values of the late-fusion policy step
    struct PackSet {                // blocks of the world kernel for one (packing, staging) choice
        int cap, budget;            // agents per block (0: one world), staged bytes per block (0: off)
        int4* d;
        int n;
    };
    std::vector<PackSet> packsets;
    int pack_cap = 32;
    unsigned long long wait_ns = 0;   // staging-wait limit of the step kernels (0: 1 s)
    int withhold = 0;                 // set up the staging barrier but issue no copy (timeout tests)
    StepScratch sc{};           // scratch of the split step
    bool loaded = false;
    unsigned gen = 0;           // bumped when a captured step would go stale (roads, launch shape)
    struct HostStep {           // the captured step of sf_step_host: copy in, step, copies out
        float dt = 0.f;
        int substeps = 0;
        unsigned gen = 0;
        const float* ha = nullptr;
        float* hr = nullptr;
        uint8_t* hd = nullptr;
        float* ho = nullptr;    // observations [A][320] (sf_step_host_obs), null: not copied
        float* d_act = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        // mapped: the step's own kernels read the actions and write rewards and
        // done flags through the buffers' device mapping (their arguments `wa`
        // are rewritten to retarget the graph); else copy nodes move them
        bool mapped = false;
        WorldArgs wa{};
        static constexpr int kMaxStepNodes = 8;
        cudaGraphNode_t n_step[kMaxStepNodes] = {};                            // kernel nodes (mapped)
        cudaKernelNodeParams kp_step[kMaxStepNodes] = {};                     // their launch parameters
        int n_steps = 0;
        cudaGraphNode_t n_act = nullptr, n_rew = nullptr, n_done = nullptr;   // copy nodes (not mapped)
        cudaGraphNode_t n_obs = nullptr;                                        // observation copy node
    } hs;
};

struct sf_graph {
    sf_ctx* h = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;           // kernels per replay
};

namespace {

sf_status fail(sf_ctx* h, sf_status s, const std::string& msg) {
    if (h) h->err = msg;
    return s;
}

sf_status cuda_fail(sf_ctx* h, cudaError_t e, const char* where) {
    return fail(h, e == cudaErrorMemoryAllocation ? SF_ERR_OOM : SF_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

#define SF_CUDA(h, call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

template <class T>
sf_status dalloc(sf_ctx* h, T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc");
    h->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return SF_OK;
}

void drop_host_step(sf_ctx* h) {
    if (h->hs.exec) cudaGraphExecDestroy(h->hs.exec);
    if (h->hs.graph) cudaGraphDestroy(h->hs.graph);
    float* d_act = h->hs.d_act;   // in h->allocs
    h->hs = sf_ctx::HostStep{};
    h->hs.d_act = d_act;
}

void free_all(sf_ctx* h) {
    drop_host_step(h);
    h->hs.d_act = nullptr;
    ++h->gen;
    if (h->surr) { ::operator delete(h->surr); h->surr = nullptr; }
    if (h->lfb) { ::operator delete(h->lfb); h->lfb = nullptr; }
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
    h->st = DevState{};
    h->rd = DevRoads{};
    h->out = DevOutputs{};
    h->place_buf = nullptr;
    h->all_mask = nullptr;
    h->act_buf = nullptr;
    h->m_epmax = nullptr;
    h->m_epev = nullptr;
    h->m_cnt = nullptr;
    h->surr = nullptr;
    h->lfb = nullptr;
    h->packsets.clear();
    h->sc = StepScratch{};
    h->loaded = false;
    h->W = h->A = h->NP = 0;
}

// ---- episode metrics (Sec. 4): success rate (episodes that reach their goal),
// collision rate (episodes with inter-vehicle contact, the collision event),
// mean episode-maximum DRAC and the share of episodes above 3.4 m/s^2, over the
// episodes ended since the counters were last cleared.  One thread per agent
// after each step: the running maximum of the step DRAC and the union of the
// step's event bits; a done agent's episode goes into the counters (integer
// atomics, block sums first, so the totals do not depend on the order), the
// DRAC sum in fixed point of 1e-6 m/s^2.
__global__ void __launch_bounds__(256) metrics_kernel(const uint32_t* __restrict__ events,
                                                      const uint8_t* __restrict__ done,
                                                      const float* __restrict__ drac, int A, float* __restrict__ epmax,
                                                      uint32_t* __restrict__ epev, unsigned long long* __restrict__ cnt) {
    __shared__ unsigned long long part[8][kMetricCount];
    const int a = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long v[kMetricCount];
#pragma unroll
    for (int i = 0; i < kMetricCount; ++i) v[i] = 0ull;
    if (a < A) {
        const float d = drac[a];
        float m = epmax[a];
        if (d > m) m = d;                               // NaN never raises the maximum
        uint32_t e = epev[a] | events[a];
        if (done[a]) {
            v[kMetricEpisodes] = 1ull;
            v[kMetricGoals] = (e & sfk::kEvGoal) ? 1ull : 0ull;
            v[kMetricCollisions] = (e & sfk::kEvCollision) ? 1ull : 0ull;
            v[kMetricCrashes] = (e & sfk::kEvCrash) ? 1ull : 0ull;
            v[kMetricOffroad] = (e & sfk::kEvOffroad) ? 1ull : 0ull;
            v[kMetricLaneForb] = (e & sfk::kEvLaneForb) ? 1ull : 0ull;
            v[kMetricIdle] = (e & sfk::kEvIdle) ? 1ull : 0ull;
            v[kMetricTimeouts] = (e & sfk::kEvTimeout) ? 1ull : 0ull;
            v[kMetricNonfinite] = (e & sfk::kEvNonfinite) ? 1ull : 0ull;
            v[kMetricDracOver] = m > 3.4f ? 1ull : 0ull;
            v[kMetricDracMicro] = (unsigned long long)llrint((double)fminf(m, 1e6f) * 1e6);
            m = 0.f;
            e = 0u;
        }
        epmax[a] = m;
        epev[a] = e;
    }
#pragma unroll
    for (int i = 0; i < kMetricCount; ++i) {
        unsigned long long x = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
        if (lane == 0) part[warp][i] = x;
    }
    __syncthreads();
    if (threadIdx.x < kMetricCount) {
        unsigned long long x = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += part[w][threadIdx.x];
        if (x) atomicAdd(cnt + threadIdx.x, x);
    }
}

// a masked reset starts new episodes: their running maxima and event bits are dropped
__global__ void metrics_reset_kernel(const uint8_t* __restrict__ mask, int A, float* __restrict__ epmax,
                                     uint32_t* __restrict__ epev) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < A && mask[a]) { epmax[a] = 0.f; epev[a] = 0u; }
}

// the metrics pass after a step (nothing without SF_FLAG_METRICS)
cudaError_t launch_metrics(const sf_ctx* h) {
    if (!h->m_cnt || h->A <= 0) return cudaSuccess;
    metrics_kernel<<<(h->A + 255) / 256, 256, 0, h->stream>>>(h->out.events, h->out.done, h->out.drac, h->A,
                                                             h->m_epmax, h->m_epev, h->m_cnt);
    return cudaGetLastError();
}

WorldArgs make_args(sf_ctx* h) {
    WorldArgs a{};
    a.st = h->st;
    a.rd = h->rd;
    a.out = h->out;
    a.num_worlds = h->W;
    a.num_agents = h->A;
    const int cap = h->cfg.pack_agents > 0 ? h->pack_cap : 0;
    const int budget = h->cfg.split_step ? 0 : h->cfg.stage_bytes;   // the split step does not stage
    for (const auto& ps : h->packsets)
        if (ps.cap == cap && ps.budget == budget) {
            a.packs = ps.d;
            a.num_packs = ps.n;
            a.stage_bytes = ps.budget;
        }
    a.sc = h->sc;
    a.flags = h->cfg.flags | (h->cfg.weather_model == SF_WEATHER_ALL ? sfk::kFlagWeatherAll : 0);
    a.seed = h->cfg.seed;
    a.dynamics = h->cfg.dynamics;
    a.substeps = 1;
    a.h = 0.f;
    a.wait_ns = h->wait_ns;
    a.withhold = h->withhold;
    return a;
}

int wpb_of(const sf_ctx* h) {
    int w = h->cfg.warps_per_block;
    return (w == 1 || w == 2 || w == 4 || w == 8) ? w : 4;
}

// one control step in the handle's launch shape (fused kernel or split step)
cudaError_t launch_step(const sf_ctx* h, const WorldArgs& a) {
    return h->cfg.split_step ? sf_launch_step_split(a, wpb_of(h), h->stream)
                             : sf_launch_world(kModeStep, a, wpb_of(h), h->stream);
}

// blocks of the world kernel: runs of consecutive non-empty worlds whose agents
// total at most `cap` (cap 0: one world per block) and, with a staging budget,
// whose road blobs total at most `budget` bytes (a larger world gets a block
// alone and is read from global memory)
std::vector<int4> make_packs(const std::vector<int4>& world, const std::vector<DevGrid>& grid, int cap, int budget) {
    std::vector<int4> packs;
    int4 cur = make_int4(0, 0, 0, 0);
    long long bytes = 0;
    bool open = false;
    for (int w = 0; w < (int)world.size(); ++w) {
        const int n = world[w].y;
        if (n <= 0) { if (open) packs.push_back(cur); open = false; continue; }
        const long long b = grid[w].bytes;
        if (open && (cap <= 0 || cur.w + n > cap || (budget > 0 && bytes + b > budget))) {
            packs.push_back(cur);
            open = false;
        }
        if (!open) { cur = make_int4(w, 1, world[w].x, n); bytes = b; open = true; }
        else { cur.y += 1; cur.w += n; bytes += b; }
    }
    if (open) packs.push_back(cur);
    // blocks longest first: the block scheduler starts them in index order as
    // earlier ones finish, so the costliest packs do not start last (a block's
    // results do not depend on when it runs).  Estimated cycles: the physics,
    // then the road queries of its agents over its warps, each growing with
    // its world's edge segments (the edge ray tests all of them)
    auto cost = [&](const int4& p) {
        double c = 12000.0;
        for (int w = p.x; w < p.x + p.y; ++w) c += world[w].y * (7000.0 + 10.0 * grid[w].ecnt) / 8.0;
        return c;
    };
    std::stable_sort(packs.begin(), packs.end(), [&](const int4& a, const int4& b) { return cost(a) > cost(b); });
    return packs;
}

// staging budgets the autotuner tries (bytes of shared memory per block)
constexpr int kBudgets[3] = {0, 48 * 1024, 96 * 1024};

bool is_lane_type(int t) { return t == 1 || t == 2; }
bool is_edge_type(int t) { return t == 15 || t == 16; }

}  // namespace

// ---------------------------------------------------------------- dynamics surrogate objects
struct sf_surrogate {
    sf_mlp_handle mlp = nullptr;
    cudaStream_t stream = nullptr;
    float* stats = nullptr;       // [30 mean, 30 std, 16 mean, 16 std]
    float* bx = nullptr;          // training minibatch [batch][30]
    float* by = nullptr;          // [batch][16]
    int bcap = 0;
    bool trained = false;
    std::string err;
};

struct SurrBufs {                 // per-world-handle buffers of the surrogate step
    float* x = nullptr;           // [A][32] normalised features
    float* y = nullptr;           // [A][16] normalised outputs
    float4* snap = nullptr;       // [5][A]
    uint8_t* elig = nullptr;      // [A]
    unsigned* words = nullptr;    // [0] audit error bits, [1] surrogate uses
};


static SurrBufs* surr_bufs(sf_ctx* h) {
    if (h->surr) return static_cast<SurrBufs*>(h->surr);
    const size_t A = (size_t)h->A;
    SurrBufs* b = new SurrBufs();
    bool ok = dalloc(h, &b->x, A * kSurrInLd) == SF_OK && dalloc(h, &b->y, A * kSurrOut) == SF_OK &&
              dalloc(h, &b->snap, A * 5) == SF_OK && dalloc(h, &b->elig, A) == SF_OK &&
              dalloc(h, &b->words, 2) == SF_OK;
    if (!ok || cudaMemset(b->words, 0, 8) != cudaSuccess) { delete b; return nullptr; }
    h->surr = b;
    return b;
}

struct LfBufs {                   // per-world-handle buffers of the late-fusion policy step
    float* obs = nullptr;         // [A][SF_FULL_OBS_DIM]
    int32_t* n_road = nullptr;    // [A]
    int32_t* n_veh = nullptr;     // [A]
    float* value = nullptr;       // [A]
};

static LfBufs* lf_bufs(sf_ctx* h) {
    if (h->lfb) return static_cast<LfBufs*>(h->lfb);
    const size_t A = (size_t)h->A;
    LfBufs* b = new LfBufs();
    bool ok = dalloc(h, &b->obs, A * SF_FULL_OBS_DIM) == SF_OK && dalloc(h, &b->n_road, A) == SF_OK &&
              dalloc(h, &b->n_veh, A) == SF_OK && dalloc(h, &b->value, A) == SF_OK;
    if (!ok) { delete b; return nullptr; }
    h->lfb = b;
    return b;
}

cudaStream_t sf_handle_stream(sf_handle h) { return h ? h->stream : nullptr; }

extern "C" {

const char* sf_version(void) { return "sf 0.1 (sm_103a)"; }

const char* sf_last_error(sf_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

sf_status sf_create(const sf_config* cfg, void* cuda_stream, sf_handle* out) {
    g_create_error.clear();
    if (!out) { g_create_error = "sf_create: out is NULL"; return SF_ERR_INVALID_ARG; }
    *out = nullptr;
    sf_config c{};
    if (cfg) c = *cfg;
    if (c.reserved[0] != 0) { g_create_error = "sf_create: reserved fields must be zero"; return SF_ERR_INVALID_ARG; }
    if (c.weather_model != SF_WEATHER_TABLE && c.weather_model != SF_WEATHER_ALL) {
        g_create_error = "sf_create: weather_model must be SF_WEATHER_TABLE or SF_WEATHER_ALL";
        return SF_ERR_INVALID_ARG;
    }
    if (c.world_begin < 0 || c.world_end < 0 || (c.world_end != 0 && c.world_end <= c.world_begin) ||
        (c.world_end == 0 && c.world_begin != 0)) {
        g_create_error = "sf_create: world range must be 0 <= world_begin < world_end (or both 0)";
        return SF_ERR_INVALID_ARG;
    }
    if (c.dynamics != SF_DYN_VEHICLE && c.dynamics != SF_DYN_BICYCLE) {
        g_create_error = "sf_create: dynamics must be SF_DYN_VEHICLE or SF_DYN_BICYCLE";
        return SF_ERR_INVALID_ARG;
    }
    if (c.split_step != 0 && c.split_step != 1) {
        g_create_error = "sf_create: split_step must be 0 or 1";
        return SF_ERR_INVALID_ARG;
    }
    if (c.stage_bytes < 0 || c.stage_bytes > sfk::kMaxStageBytes || c.stage_bytes % 16) {
        g_create_error = "sf_create: stage_bytes must be a multiple of 16 in 0..163840";
        return SF_ERR_INVALID_ARG;
    }
    if (c.pack_agents < 0 || c.pack_agents > 32) {
        g_create_error = "sf_create: pack_agents must be 0..32";
        return SF_ERR_INVALID_ARG;
    }
    int dev = 0, count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        g_create_error = std::string("sf_create: no CUDA device: ") + cudaGetErrorString(e);
        return SF_ERR_CUDA;
    }
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { g_create_error = cudaGetErrorString(e); return SF_ERR_CUDA; }
    sf_ctx* h = new sf_ctx();
    h->cfg = c;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->device = dev;
    *out = h;
    return SF_OK;
}

sf_status sf_destroy(sf_handle h) {
    if (!h) return SF_OK;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return SF_OK;
}

int32_t sf_num_agents(sf_handle h) { return h ? h->A : 0; }
int32_t sf_num_worlds(sf_handle h) { return h ? h->W : 0; }

sf_status sf_load_roads(sf_handle h, const sf_roads* r) {
    if (!h) return SF_ERR_INVALID_ARG;
    if (!r) return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: roads is NULL");
    // world range: the CSR of worlds [world_begin, world_end), offsets re-based
    sf_roads rs{};
    std::vector<int32_t> s_aoff, s_poff, s_ptoff;
    int agent_base = 0;
    if (h->cfg.world_end != 0) {
        const int w0 = h->cfg.world_begin, w1 = h->cfg.world_end;
        if (w1 > r->num_worlds) return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: world range beyond num_worlds");
        if (!r->agent_off || !r->poly_off || !r->point_off)
            return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: NULL array");
        const int a0 = r->agent_off[w0], p0 = r->poly_off[w0], p1 = r->poly_off[w1];
        if (a0 < 0 || p0 < 0 || p1 < p0 || p1 > r->num_polylines)
            return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: world range offsets out of order");
        const int q0 = r->point_off[p0];
        if (q0 < 0 || r->point_off[p1] < q0)
            return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: world range offsets out of order");
        for (int w = w0; w <= w1; ++w) {
            s_aoff.push_back(r->agent_off[w] - a0);
            s_poff.push_back(r->poly_off[w] - p0);
        }
        for (int p = p0; p <= p1; ++p) s_ptoff.push_back(r->point_off[p] - q0);
        rs.num_worlds = w1 - w0;
        rs.num_polylines = p1 - p0;
        rs.num_points = r->point_off[p1] - q0;
        rs.agent_off = s_aoff.data();
        rs.poly_off = s_poff.data();
        rs.point_off = s_ptoff.data();
        rs.poly_type = r->poly_type ? r->poly_type + p0 : nullptr;
        rs.px = r->px ? r->px + q0 : nullptr;
        rs.py = r->py ? r->py + q0 : nullptr;
        rs.precip = r->precip ? r->precip + a0 : nullptr;
        rs.surface = r->surface ? r->surface + a0 : nullptr;
        rs.film_mm = r->film_mm ? r->film_mm + a0 : nullptr;
        agent_base = a0;
        r = &rs;
    }
    const int W = r->num_worlds, NPl = r->num_polylines, NP = r->num_points;
    if (W <= 0 || NPl < 0 || NP < 0) return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: negative or zero sizes");
    if (!r->agent_off || !r->poly_off || !r->point_off || (NPl > 0 && !r->poly_type) || (NP > 0 && (!r->px || !r->py)))
        return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: NULL array");
    if (r->agent_off[0] != 0 || r->poly_off[0] != 0 || r->point_off[0] != 0)
        return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: CSR offsets must start at 0");
    for (int w = 0; w < W; ++w) {
        int na = r->agent_off[w + 1] - r->agent_off[w];
        if (na < 0 || na > SF_MAX_AGENTS_PER_WORLD)
            return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: world " + std::to_string(w) + " has " +
                                                   std::to_string(na) + " agents (0..32 allowed)");
        if (r->poly_off[w + 1] < r->poly_off[w])
            return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: poly_off not monotone at world " + std::to_string(w));
    }
    if (r->poly_off[W] != NPl) return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: poly_off[W] != num_polylines");
    for (int p = 0; p < NPl; ++p)
        if (r->point_off[p + 1] < r->point_off[p])
            return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: point_off not monotone at polyline " + std::to_string(p));
    if (r->point_off[NPl] != NP) return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: point_off[P] != num_points");
    const int A = r->agent_off[W];
    const bool all_model = h->cfg.weather_model == SF_WEATHER_ALL;
    if (A > 0 && (!r->surface || (all_model ? !r->film_mm : !r->precip)))
        return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: NULL weather arrays");
    for (int a = 0; a < A; ++a) {
        const bool bad = all_model ? !(std::isfinite(r->film_mm[a]) && r->film_mm[a] >= 0.f) : r->precip[a] > 3;
        if (bad || r->surface[a] > 2)
            return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: weather code out of range at agent " + std::to_string(a));
    }
    for (int k = 0; k < NP; ++k)
        if (!std::isfinite(r->px[k]) || !std::isfinite(r->py[k]))
            return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: non-finite point " + std::to_string(k));

    // ---- derived road store (double precision on the host, App. C rules)
    std::vector<float4> pt(NP);
    std::vector<uint32_t> pmeta(NP);
    std::vector<int32_t> pend(NP);
    std::vector<int4> world(W);
    std::vector<int2> cand(W);
    std::vector<int32_t> cands;
    std::vector<DevGrid> grid(W);
    std::vector<int32_t> pbeg(NP);
    std::vector<float> arcl(NP);
    std::vector<float4> mid(NP);       // segment k -> k+1: midpoint (double, rounded) and unit direction
    std::vector<uint8_t> ptype(NP);
    std::vector<unsigned char> blob;   // every world's road blob, 16-byte aligned sections
    auto in_box = [](double x, double y) { return std::fabs(x) <= 100.0 && std::fabs(y) <= 100.0; };
    for (int w = 0; w < W; ++w) {
        const int p0 = r->poly_off[w], p1 = r->poly_off[w + 1];
        const int q0 = r->point_off[p0], q1 = r->point_off[p1];
        world[w] = make_int4(r->agent_off[w], r->agent_off[w + 1] - r->agent_off[w], q0, q1 - q0);
        std::vector<int32_t> strict, all_lane;
        for (int p = p0; p < p1; ++p) {
            const int t = r->poly_type[p];
            const int k0 = r->point_off[p], k1 = r->point_off[p + 1];
            std::vector<double> arc(k1 - k0, 0.0);
            for (int k = k0; k < k1; ++k) {
                if (k > k0) {
                    double dx = (double)r->px[k] - r->px[k - 1], dy = (double)r->py[k] - r->py[k - 1];
                    arc[k - k0] = arc[k - k0 - 1] + std::sqrt(dx * dx + dy * dy);
                }
                int a = -1, b = -1;
                if (k + 1 < k1) { a = k; b = k + 1; } else if (k - 1 >= k0) { a = k - 1; b = k; }
                double dxn = 0, dyn = 0;
                if (a >= 0) {
                    double dx = (double)r->px[b] - r->px[a], dy = (double)r->py[b] - r->py[a];
                    double n = std::sqrt(dx * dx + dy * dy);
                    if (n > 0) { dxn = dx / n; dyn = dy / n; }
                }
                pt[k] = make_float4(r->px[k], r->py[k], (float)dxn, (float)dyn);
                uint32_t m = (uint32_t)t & sfk::kPtTypeMask;
                if (k + 1 < k1) {
                    double dx = (double)r->px[k + 1] - r->px[k], dy = (double)r->py[k + 1] - r->py[k];
                    if (std::sqrt(dx * dx + dy * dy) <= 3.0 && in_box(r->px[k], r->py[k]) &&
                        in_box(r->px[k + 1], r->py[k + 1]))
                        m |= sfk::kPtSegNext;
                }
                if (is_lane_type(t)) m |= sfk::kPtLane;
                if (is_edge_type(t)) m |= sfk::kPtEdge;
                pmeta[k] = m;
                ptype[k] = (uint8_t)t;
                mid[k] = make_float4(INFINITY, 0.f, 0.f, 0.f);
                if (m & sfk::kPtSegNext) {
                    const double ax = r->px[k], ay = r->py[k], bx = r->px[k + 1], by = r->py[k + 1];
                    const double n = std::sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
                    mid[k] = make_float4((float)(0.5 * (ax + bx)), (float)(0.5 * (ay + by)),
                                         n > 0 ? (float)((bx - ax) / n) : 0.f, n > 0 ? (float)((by - ay) / n) : 0.f);
                }
                pend[k] = k1;
                pbeg[k] = k0;
                arcl[k] = (float)arc[k - k0];
            }
            if (is_lane_type(t) && k1 > k0) {
                const double total = arc.back();
                for (int k = k0; k < k1; ++k) {
                    all_lane.push_back(k);
                    if (total - arc[k - k0] >= 50.0) strict.push_back(k);
                }
            }
        }
        const std::vector<int32_t>& use = strict.empty() ? all_lane : strict;
        cand[w] = make_int2((int)cands.size(), (int)use.size());
        cands.insert(cands.end(), use.begin(), use.end());

        // ---- the world's road blob: grid cell offsets, cell-sorted segment
        // records (row-major cells, input order within a cell), info words, edges
        if (q1 - q0 > sfk::kMaxWorldPoints)
            return fail(h, SF_ERR_INVALID_ARG, "sf_load_roads: world " + std::to_string(w) + " has " +
                                                   std::to_string(q1 - q0) + " road points (at most 65535)");
        double xmin = 0, xmax = 0, ymin = 0, ymax = 0;
        for (int k = q0; k < q1; ++k) {
            if (k == q0 || r->px[k] < xmin) xmin = r->px[k];
            if (k == q0 || r->px[k] > xmax) xmax = r->px[k];
            if (k == q0 || r->py[k] < ymin) ymin = r->py[k];
            if (k == q0 || r->py[k] > ymax) ymax = r->py[k];
        }
        double c = std::max(sfk::kCellMin, std::max(xmax - xmin, ymax - ymin) / (sfk::kGridMax - 1));
        int nx = std::min(sfk::kGridMax, (int)std::floor((xmax - xmin) / c) + 1);
        int ny = std::min(sfk::kGridMax, (int)std::floor((ymax - ymin) / c) + 1);
        const int ncell = nx * ny, np = q1 - q0;
        auto cx_of = [&](double x) { return std::min(nx - 1, std::max(0, (int)std::floor((x - xmin) / c))); };
        auto cy_of = [&](double y) { return std::min(ny - 1, std::max(0, (int)std::floor((y - ymin) / c))); };
        std::vector<int> cnt(ncell + 1, 0);
        std::vector<float4> edges;
        for (int k = q0; k < q1; ++k) {
            cnt[cy_of(r->py[k]) * nx + cx_of(r->px[k]) + 1]++;
            if ((pmeta[k] & (sfk::kPtSegNext | sfk::kPtEdge)) == (sfk::kPtSegNext | sfk::kPtEdge))
                edges.push_back(make_float4(r->px[k], r->py[k], r->px[k + 1], r->py[k + 1]));
        }
        for (int i = 0; i < ncell; ++i) cnt[i + 1] += cnt[i];
        // the edges sorted (stable) by the cell of their start point in the coarse edge grid
        const double ce = std::max(sfk::kEdgeCellMin, std::max(xmax - xmin, ymax - ymin) / (sfk::kEdgeGridMax - 1));
        const int ex = std::min(sfk::kEdgeGridMax, (int)std::floor((xmax - xmin) / ce) + 1);
        const int ey = std::min(sfk::kEdgeGridMax, (int)std::floor((ymax - ymin) / ce) + 1);
        auto ecell = [&](const float4& e) {
            const int cx = std::min(ex - 1, std::max(0, (int)std::floor((e.x - xmin) / ce)));
            const int cy = std::min(ey - 1, std::max(0, (int)std::floor((e.y - ymin) / ce)));
            return cy * ex + cx;
        };
        std::vector<int> ecnt_c(ex * ey + 1, 0);
        for (const float4& e : edges) ecnt_c[ecell(e) + 1]++;
        for (int i = 0; i < ex * ey; ++i) ecnt_c[i + 1] += ecnt_c[i];
        {
            std::vector<float4> sorted(edges.size());
            std::vector<int> pos(ecnt_c.begin(), ecnt_c.end() - 1);
            for (const float4& e : edges) sorted[pos[ecell(e)]++] = e;
            edges.swap(sorted);
        }
        auto a16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
        const size_t o_seg = a16(2 * (size_t)(ncell + 1)), o_info = o_seg + 16 * (size_t)np,
                     o_edge = o_info + a16(4 * (size_t)np), o_eoff = o_edge + 16 * edges.size(),
                     bytes = a16(o_eoff + 2 * (size_t)(ex * ey + 1));
        const size_t at = blob.size();
        blob.resize(at + bytes, 0);
        unsigned char* B = blob.data() + at;
        for (int i = 0; i <= ncell; ++i) {
            const uint16_t v = (uint16_t)cnt[i];
            std::memcpy(B + 2 * i, &v, 2);
        }
        for (int k = q0; k < q1; ++k) {   // stable: input order within a cell
            const int slot = cnt[cy_of(r->py[k]) * nx + cx_of(r->px[k])]++;
            const bool has_next = k + 1 < pend[k];
            const int o = has_next ? k + 1 : (k - 1 >= pbeg[k] ? k - 1 : k);
            const float4 rec = make_float4(r->px[k], r->py[k], r->px[o], r->py[o]);
            uint32_t info = (uint32_t)(k - q0) | ((pmeta[k] & sfk::kPtTypeMask) << 16);
            if (pmeta[k] & sfk::kPtSegNext) info |= sfk::kInfoSegNext;
            if (pmeta[k] & sfk::kPtLane) info |= sfk::kInfoLane;
            if (pmeta[k] & sfk::kPtEdge) info |= sfk::kInfoEdge;
            if (has_next) info |= sfk::kInfoHasNext;
            std::memcpy(B + o_seg + 16 * (size_t)slot, &rec, 16);
            std::memcpy(B + o_info + 4 * (size_t)slot, &info, 4);
        }
        if (!edges.empty()) std::memcpy(B + o_edge, edges.data(), 16 * edges.size());
        for (int i = 0; i <= ex * ey; ++i) {
            const uint16_t v = (uint16_t)ecnt_c[i];
            std::memcpy(B + o_eoff + 2 * i, &v, 2);
        }
        DevGrid g{};
        g.inv_ce = (float)(1.0 / ce); g.ex = ex; g.ey = ey; g.o_eoff = (int)o_eoff;
        g.x0 = (float)xmin; g.y0 = (float)ymin; g.c = (float)c; g.inv_c = (float)(1.0 / c);
        g.nx = nx; g.ny = ny; g.np = np; g.ecnt = (int)edges.size();
        g.bytes = (int)bytes; g.o_seg = (int)o_seg; g.o_info = (int)o_info; g.o_edge = (int)o_edge;
        g.q0 = q0;
        g.blob = at;
        grid[w] = g;
    }

    // ---- allocate and upload
    cudaStreamSynchronize(h->stream);
    free_all(h);
    sf_status s;
    const size_t Aa = (size_t)A;
#define SF_ALLOC(ptr, T, n) \
    if ((s = dalloc(h, &(ptr), (n))) != SF_OK) { free_all(h); return s; }
    float4 *pos, *quat, *vel, *angv, *spin, *goal;
    SF_ALLOC(pos, float4, Aa);
    SF_ALLOC(quat, float4, Aa);
    SF_ALLOC(vel, float4, Aa);
    SF_ALLOC(angv, float4, Aa);
    SF_ALLOC(spin, float4, Aa);
    SF_ALLOC(goal, float4, Aa);
    float* peak; uint32_t* meta; int32_t *step, *episode;
    SF_ALLOC(peak, float, Aa);
    SF_ALLOC(meta, uint32_t, Aa);
    SF_ALLOC(step, int32_t, Aa);
    SF_ALLOC(episode, int32_t, Aa);
    h->st = DevState{pos, quat, vel, angv, spin, goal, peak, meta, step, episode};
    int4* dworld; int2* dcand; float4* dpt; int32_t *dpend, *dcands; float* darc;
    SF_ALLOC(dworld, int4, (size_t)W);
    SF_ALLOC(dcand, int2, (size_t)W);
    SF_ALLOC(dpt, float4, (size_t)NP + 1);
    SF_ALLOC(dpend, int32_t, (size_t)NP + 1);
    SF_ALLOC(darc, float, (size_t)NP + 1);
    SF_ALLOC(dcands, int32_t, cands.size() + 1);
    DevGrid* dgrid; unsigned char* dblob;
    SF_ALLOC(dgrid, DevGrid, (size_t)W);
    SF_ALLOC(dblob, unsigned char, blob.size() + 16);
    float4* dmid; uint8_t* dptype;
    SF_ALLOC(dmid, float4, (size_t)NP + 1);
    SF_ALLOC(dptype, uint8_t, (size_t)NP + 1);
    // spawn table (one entry per spawn candidate) and each candidate's world, for its build
    const int ncand = (int)cands.size();
    SpawnQ* dspawnq; int32_t* dcand_world;
    SF_ALLOC(dspawnq, SpawnQ, (size_t)ncand + 1);
    SF_ALLOC(dcand_world, int32_t, (size_t)ncand + 1);
    h->rd = DevRoads{dworld, dcand, dpt, dpend, darc, dcands, dgrid, dblob, dmid, dptype, agent_base, dspawnq};
    float *obs, *reward, *drac; uint8_t* done; uint32_t* events; int32_t *lane_seg, *knn_pts, *knn_agents;
    unsigned int* err_word; float* hint;
    SF_ALLOC(obs, float, Aa * SF_OBS_DIM);
    SF_ALLOC(reward, float, Aa);
    SF_ALLOC(done, uint8_t, Aa);
    SF_ALLOC(events, uint32_t, Aa);
    SF_ALLOC(lane_seg, int32_t, Aa);
    SF_ALLOC(knn_pts, int32_t, Aa * SF_L_POINTS);
    SF_ALLOC(knn_agents, int32_t, Aa * SF_K_AGENTS);
    SF_ALLOC(drac, float, Aa);
    SF_ALLOC(err_word, unsigned int, 1);
    SF_ALLOC(hint, float, Aa * 4);
    h->out = DevOutputs{obs, reward, done, events, lane_seg, knn_pts, knn_agents, drac, err_word, hint};
    SF_ALLOC(h->place_buf, float, Aa * 6);
    SF_ALLOC(h->all_mask, uint8_t, Aa);
    SF_ALLOC(h->act_buf, float, Aa * 3);
    AgentQ* scq; float2 *scprev, *schead; uint8_t* scflag; int32_t *scworld, *scfix; unsigned* sccount;
    SF_ALLOC(scq, AgentQ, Aa);
    SF_ALLOC(scprev, float2, Aa);
    SF_ALLOC(schead, float2, Aa);
    SF_ALLOC(scflag, uint8_t, Aa);
    SF_ALLOC(scworld, int32_t, Aa);
    SF_ALLOC(scfix, int32_t, Aa);
    SF_ALLOC(sccount, unsigned, 1);
    h->sc = StepScratch{scq, scprev, schead, scflag, scworld, scfix, sccount};
    std::vector<int32_t> agent_world(Aa);
    for (int w = 0; w < W; ++w)
        for (int k = world[w].x; k < world[w].x + world[w].y; ++k) agent_world[k] = w;
    h->pack_cap = h->cfg.pack_agents > 0 ? h->cfg.pack_agents : 32;
    std::vector<int> budgets(kBudgets, kBudgets + 3);
    if (std::find(budgets.begin(), budgets.end(), h->cfg.stage_bytes) == budgets.end())
        budgets.push_back(h->cfg.stage_bytes);
    std::vector<std::vector<int4>> pack_host;
    for (int budget : budgets)
        for (int cap : {0, h->pack_cap}) {
            pack_host.push_back(make_packs(world, grid, cap, budget));
            sf_ctx::PackSet ps{cap, budget, nullptr, (int)pack_host.back().size()};
            SF_ALLOC(ps.d, int4, pack_host.back().size());
            h->packsets.push_back(ps);
        }
    if (h->cfg.flags & SF_FLAG_METRICS) {
        SF_ALLOC(h->m_epmax, float, Aa);
        SF_ALLOC(h->m_epev, uint32_t, Aa);
        SF_ALLOC(h->m_cnt, unsigned long long, kMetricCount);
    }
#undef SF_ALLOC

    std::vector<uint32_t> meta_h(Aa);
    // the weather byte: the precipitation class, or (ALL model) the water film in
    // hundredths of a millimetre, held to 2.55 mm (mu is the floor beyond 0.85 mm)
    for (size_t a = 0; a < Aa; ++a) {
        const uint32_t wb = all_model ? (uint32_t)std::min(255.0, std::nearbyint((double)r->film_mm[a] * 100.0))
                                      : (uint32_t)r->precip[a];
        meta_h[a] = wb | ((uint32_t)r->surface[a] << 8);
    }
    cudaError_t e = cudaSuccess;
    auto up = [&](void* d, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice);
    };
    auto zero = [&](void* d, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemset(d, 0, bytes);
    };
    up(dworld, world.data(), world.size() * sizeof(int4));
    up(dcand, cand.data(), cand.size() * sizeof(int2));
    up(dpt, pt.data(), pt.size() * sizeof(float4));
    up(dpend, pend.data(), pend.size() * sizeof(int32_t));
    up(darc, arcl.data(), arcl.size() * sizeof(float));
    up(dcands, cands.data(), cands.size() * sizeof(int32_t));
    up(dgrid, grid.data(), grid.size() * sizeof(DevGrid));
    up(dblob, blob.data(), blob.size());
    up(dmid, mid.data(), mid.size() * sizeof(float4));
    up(dptype, ptype.data(), ptype.size());
    for (float4* p : {pos, quat, vel, angv, spin, goal}) zero(p, Aa * sizeof(float4));
    zero(peak, Aa * 4); zero(step, Aa * 4); zero(episode, Aa * 4);
    up(meta, meta_h.data(), Aa * 4);
    up(scworld, agent_world.data(), Aa * 4);
    zero(scflag, Aa);
    zero(sccount, 4);
    zero(obs, Aa * SF_OBS_DIM * 4); zero(reward, Aa * 4); zero(done, Aa); zero(events, Aa * 4);
    zero(drac, Aa * 4); zero(err_word, 4); zero(hint, Aa * 16);
    if (h->m_cnt) { zero(h->m_epmax, Aa * 4); zero(h->m_epev, Aa * 4); zero(h->m_cnt, kMetricCount * 8); }
    if (e == cudaSuccess && Aa) e = cudaMemset(lane_seg, 0xFF, Aa * 4);
    if (e == cudaSuccess && Aa) e = cudaMemset(knn_pts, 0xFF, Aa * SF_L_POINTS * 4);
    if (e == cudaSuccess && Aa) e = cudaMemset(knn_agents, 0xFF, Aa * SF_K_AGENTS * 4);
    if (e == cudaSuccess && Aa) e = cudaMemset(h->all_mask, 1, Aa);
    for (size_t i = 0; i < h->packsets.size(); ++i)
        up(h->packsets[i].d, pack_host[i].data(), pack_host[i].size() * sizeof(int4));
    // the spawn table: the road answers at every spawn candidate, by the step's exact queries
    std::vector<int32_t> cand_world(ncand);
    for (int w = 0; w < W; ++w)
        for (int k = cand[w].x; k < cand[w].x + cand[w].y; ++k) cand_world[k] = w;
    up(dcand_world, cand_world.data(), (size_t)ncand * 4);
    if (e == cudaSuccess) e = sf_launch_spawn_table(h->rd, dcand_world, ncand, dspawnq, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { free_all(h); return cuda_fail(h, e, "sf_load_roads upload"); }
    h->W = W; h->A = A; h->NP = NP;
    h->loaded = true;
    return SF_OK;
}

sf_status sf_step(sf_handle h, const float* d_actions, float dt, int substeps) {
    if (!h) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_step: no roads loaded");
    if (!d_actions && h->A > 0) return fail(h, SF_ERR_INVALID_ARG, "sf_step: actions is NULL");
    if (!(dt > 0.f) || !std::isfinite(dt)) return fail(h, SF_ERR_INVALID_ARG, "sf_step: dt must be > 0");
    if (substeps < 1 || substeps > 64) return fail(h, SF_ERR_INVALID_ARG, "sf_step: substeps must be 1..64");
    WorldArgs a = make_args(h);
    a.actions = d_actions;
    a.h = dt / (float)substeps;
    a.substeps = substeps;
    cudaError_t e = launch_step(h, a);
    if (e == cudaSuccess) e = launch_metrics(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "sf_step launch");
    return SF_OK;
}

namespace {

// the device address of a page-locked host buffer, or null when it has none
void* device_view(const void* p) {
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, const_cast<void*>(p), 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return d;
}

bool page_locked(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

// the transfer nodes of a captured host step: the step's kernel nodes (mapped
// buffers; every kernel of the step takes the one WorldArgs) or the copy nodes,
// told apart by their host pointers
void find_copy_nodes(sf_ctx* h) {
    size_t n = 0;
    cudaGraphGetNodes(h->hs.graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    cudaGraphGetNodes(h->hs.graph, nodes.data(), &n);
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) != cudaSuccess) continue;
        if (t == cudaGraphNodeTypeKernel) {
            cudaKernelNodeParams mk{};
            if (cudaGraphKernelNodeGetParams(nd, &mk) == cudaSuccess &&
                mk.func == reinterpret_cast<void*>(metrics_kernel))
                continue;   // the metrics pass reads only device outputs
            const int i = h->hs.n_steps++;   // more than kMaxStepNodes: not retargeted (re-captured)
            if (i < sf_ctx::HostStep::kMaxStepNodes) {
                h->hs.n_step[i] = nd;
                cudaKernelNodeParams kp{};
                if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) h->hs.n_steps = sf_ctx::HostStep::kMaxStepNodes + 1;
                kp.kernelParams = nullptr;
                kp.extra = nullptr;
                h->hs.kp_step[i] = kp;
            }
            continue;
        }
        if (t != cudaGraphNodeTypeMemcpy) continue;
        cudaMemcpy3DParms prm{};
        if (cudaGraphMemcpyNodeGetParams(nd, &prm) != cudaSuccess) continue;
        if (prm.srcPtr.ptr == h->hs.ha) h->hs.n_act = nd;
        else if (prm.dstPtr.ptr == h->hs.hr) h->hs.n_rew = nd;
        else if (prm.dstPtr.ptr == h->hs.hd) h->hs.n_done = nd;
        else if (h->hs.ho && prm.dstPtr.ptr == h->hs.ho) h->hs.n_obs = nd;
    }
}

// the control step from host buffers (sf_step_host, and with h_obs sf_step_host_obs)
sf_status step_host(sf_handle h, const float* h_actions, float* h_obs, float* h_reward, uint8_t* h_done, float dt,
                    int substeps) {
    if (!h) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_step_host: no roads loaded");
    if (h->A > 0 && (!h_actions || !h_reward || !h_done)) return fail(h, SF_ERR_INVALID_ARG, "sf_step_host: NULL buffer");
    if (!(dt > 0.f) || !std::isfinite(dt)) return fail(h, SF_ERR_INVALID_ARG, "sf_step_host: dt must be > 0");
    if (substeps < 1 || substeps > 64) return fail(h, SF_ERR_INVALID_ARG, "sf_step_host: substeps must be 1..64");
    const size_t A = (size_t)h->A;
    sf_ctx::HostStep& c = h->hs;
    if (!c.d_act) {
        void* p = nullptr;
        SF_CUDA(h, cudaMalloc(&p, A * 12 + 16));
        h->allocs.push_back(p);
        c.d_act = static_cast<float*>(p);
    }
    const size_t obs_bytes = A * SF_OBS_DIM * 4;
    // the graph copies the observation or not: a change of that re-captures
    const bool same = c.exec && c.dt == dt && c.substeps == substeps && c.gen == h->gen &&
                      (c.ho != nullptr) == (h_obs != nullptr);
    if (same && c.ha == h_actions && c.hr == h_reward && c.hd == h_done && c.ho == h_obs) {   // replay
        SF_CUDA(h, cudaGraphLaunch(c.exec, h->stream));
        SF_CUDA(h, cudaStreamSynchronize(h->stream));
        return SF_OK;
    }
    // buffers with a device address are page-locked (and mapped): only the others
    // need the pointer query
    const float* da = A > 0 ? static_cast<const float*>(device_view(h_actions)) : nullptr;
    float* dr = A > 0 ? static_cast<float*>(device_view(h_reward)) : nullptr;
    uint8_t* dd = A > 0 ? static_cast<uint8_t*>(device_view(h_done)) : nullptr;
    const bool mapped = da && dr && dd;
    const bool pinned = (mapped || (page_locked(h_actions) && page_locked(h_reward) && page_locked(h_done))) &&
                        (!h_obs || page_locked(h_obs));
    if (!h->stream || !pinned || A == 0) {   // no graph: plain copies around the step
        if (A > 0) SF_CUDA(h, cudaMemcpyAsync(c.d_act, h_actions, A * 12, cudaMemcpyHostToDevice, h->stream));
        sf_status st = sf_step(h, c.d_act, dt, substeps);
        if (st != SF_OK) return st;
        if (A > 0) {
            SF_CUDA(h, cudaMemcpyAsync(h_reward, h->out.reward, A * 4, cudaMemcpyDeviceToHost, h->stream));
            SF_CUDA(h, cudaMemcpyAsync(h_done, h->out.done, A, cudaMemcpyDeviceToHost, h->stream));
            if (h_obs) SF_CUDA(h, cudaMemcpyAsync(h_obs, h->out.obs, obs_bytes, cudaMemcpyDeviceToHost, h->stream));
        }
        SF_CUDA(h, cudaStreamSynchronize(h->stream));
        return SF_OK;
    }
    // page-locked buffers with device addresses are read and written by the
    // step's kernels themselves (loads and posted stores over the host link);
    // others get copy nodes
    if (same && c.mapped == mapped && (!h_obs || c.n_obs)) {   // other buffers: retarget the graph's transfers
        if (h_obs)
            SF_CUDA(h, cudaGraphExecMemcpyNodeSetParams1D(c.exec, c.n_obs, h_obs, h->out.obs, obs_bytes,
                                                          cudaMemcpyDeviceToHost));
        if (mapped && c.n_steps > 0 && c.n_steps <= sf_ctx::HostStep::kMaxStepNodes) {
            c.wa.actions = da;
            c.wa.host_reward = dr;
            c.wa.host_done = dd;
            for (int i = 0; i < c.n_steps; ++i) {
                cudaKernelNodeParams kp = c.kp_step[i];   // as captured (function, grid, block, shared memory)
                void* step_args[] = {&c.wa};
                kp.kernelParams = step_args;
                kp.extra = nullptr;
                SF_CUDA(h, cudaGraphExecKernelNodeSetParams(c.exec, c.n_step[i], &kp));
            }
        } else if (!mapped && c.n_act && c.n_rew && c.n_done) {
            SF_CUDA(h, cudaGraphExecMemcpyNodeSetParams1D(c.exec, c.n_act, c.d_act, h_actions, A * 12,
                                                          cudaMemcpyHostToDevice));
            SF_CUDA(h, cudaGraphExecMemcpyNodeSetParams1D(c.exec, c.n_rew, h_reward, h->out.reward, A * 4,
                                                          cudaMemcpyDeviceToHost));
            SF_CUDA(h, cudaGraphExecMemcpyNodeSetParams1D(c.exec, c.n_done, h_done, h->out.done, A,
                                                          cudaMemcpyDeviceToHost));
        } else {
            goto capture;
        }
        c.ha = h_actions; c.hr = h_reward; c.hd = h_done; c.ho = h_obs;
        SF_CUDA(h, cudaGraphLaunch(c.exec, h->stream));
        SF_CUDA(h, cudaStreamSynchronize(h->stream));
        return SF_OK;
    }
capture:
    drop_host_step(h);
    SF_CUDA(h, cudaStreamSynchronize(h->stream));
    SF_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    sf_status st = SF_OK;
    if (mapped) {   // the step's kernels on the host buffers (fused: one node; split: four)
        c.wa = make_args(h);
        c.wa.actions = da;
        c.wa.h = dt / (float)substeps;
        c.wa.substeps = substeps;
        c.wa.host_reward = dr;
        c.wa.host_done = dd;
        e = launch_step(h, c.wa);
        if (e == cudaSuccess) e = launch_metrics(h);
        if (e != cudaSuccess) st = SF_ERR_CUDA;
    } else {
        e = cudaMemcpyAsync(c.d_act, h_actions, A * 12, cudaMemcpyHostToDevice, h->stream);
        st = e == cudaSuccess ? sf_step(h, c.d_act, dt, substeps) : SF_ERR_CUDA;
        if (e == cudaSuccess && st == SF_OK) {
            e = cudaMemcpyAsync(h_reward, h->out.reward, A * 4, cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h_done, h->out.done, A, cudaMemcpyDeviceToHost, h->stream);
        }
    }
    // the observation block goes by the copy engine (1,280 B per agent)
    if (e == cudaSuccess && st == SF_OK && h_obs)
        e = cudaMemcpyAsync(h_obs, h->out.obs, obs_bytes, cudaMemcpyDeviceToHost, h->stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess || st != SF_OK) {
        if (graph) cudaGraphDestroy(graph);
        if (st != SF_OK) return st;
        return cuda_fail(h, e != cudaSuccess ? e : e2, "sf_step_host capture");
    }
    c.graph = graph;
    e = cudaGraphInstantiate(&c.exec, graph, 0);
    if (e != cudaSuccess) {
        drop_host_step(h);
        return cuda_fail(h, e, "sf_step_host instantiate");
    }
    c.dt = dt; c.substeps = substeps; c.gen = h->gen; c.mapped = mapped;
    c.ha = h_actions; c.hr = h_reward; c.hd = h_done; c.ho = h_obs;
    find_copy_nodes(h);
    SF_CUDA(h, cudaGraphLaunch(c.exec, h->stream));
    SF_CUDA(h, cudaStreamSynchronize(h->stream));
    return SF_OK;
}

}  // namespace

sf_status sf_step_host(sf_handle h, const float* h_actions, float* h_reward, uint8_t* h_done, float dt,
                       int substeps) {
    return step_host(h, h_actions, nullptr, h_reward, h_done, dt, substeps);
}

sf_status sf_step_host_obs(sf_handle h, const float* h_actions, float* h_obs, float* h_reward, uint8_t* h_done,
                           float dt, int substeps) {
    if (h && h->A > 0 && !h_obs) return fail(h, SF_ERR_INVALID_ARG, "sf_step_host_obs: NULL observation buffer");
    return step_host(h, h_actions, h_obs, h_reward, h_done, dt, substeps);
}

sf_status sf_autotune(sf_handle h, const float* d_actions, float dt, int substeps, int iters, int32_t* out_shape,
                      float* out_ms) {
    if (!h) return SF_ERR_INVALID_ARG;
    ++h->gen;   // a step captured by sf_step_host re-captures with the tuned shape
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_autotune: no roads loaded");
    if (iters < 1) return fail(h, SF_ERR_INVALID_ARG, "sf_autotune: iters must be >= 1");
    const size_t A = (size_t)h->A;
    // every buffer a step writes: state, outputs, query hints, error word
    const std::pair<void*, size_t> bufs[] = {
        {h->st.pos, A * 16}, {h->st.quat, A * 16}, {h->st.vel, A * 16}, {h->st.angv, A * 16},
        {h->st.spin, A * 16}, {h->st.goal, A * 16}, {h->st.peak_drac, A * 4}, {h->st.meta, A * 4},
        {h->st.step, A * 4}, {h->st.episode, A * 4}, {h->out.obs, A * SF_OBS_DIM * 4}, {h->out.reward, A * 4},
        {h->out.done, A}, {h->out.events, A * 4}, {h->out.lane_seg, A * 4}, {h->out.knn_pts, A * SF_L_POINTS * 4},
        {h->out.knn_agents, A * SF_K_AGENTS * 4}, {h->out.drac, A * 4}, {h->out.hint, A * 16},
        {h->out.error_word, 4}};
    size_t total = 0;
    for (const auto& b : bufs) total += (b.second + 255) & ~(size_t)255;
    char* snap = nullptr;
    cudaError_t e = cudaMalloc(&snap, total + 256);
    if (e != cudaSuccess) return cuda_fail(h, e, "sf_autotune snapshot");
    auto copy_all = [&](bool save) {
        size_t off = 0;
        cudaError_t r = cudaSuccess;
        for (const auto& b : bufs) {
            if (r == cudaSuccess && b.second)
                r = cudaMemcpyAsync(save ? snap + off : b.first, save ? b.first : snap + off, b.second,
                                    cudaMemcpyDeviceToDevice, h->stream);
            off += (b.second + 255) & ~(size_t)255;
        }
        return r;
    };
    float ms[SF_AUTOTUNE_SHAPES] = {};
    int best = wpb_of(h), best_pack = h->cfg.pack_agents, best_stage = h->cfg.stage_bytes;
    float best_ms = 0.f;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = copy_all(true);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int saved = h->cfg.warps_per_block, saved_pack = h->cfg.pack_agents, saved_stage = h->cfg.stage_bytes;
    const int budgets[4] = {kBudgets[0], kBudgets[1], kBudgets[2], h->cfg.stage_bytes};
    const int nb = std::find(kBudgets, kBudgets + 3, h->cfg.stage_bytes) == kBudgets + 3 ? 4 : 3;
    bool first = true;
    const int saved_split = h->cfg.split_step;
    int best_split = saved_split;
    for (int si = 0; si < SF_AUTOTUNE_SHAPES && e == cudaSuccess; ++si) {
        const bool split = si >= 32;
        if (!split && si >= 8 * nb) continue;
        const int k = si - 32;
        const int nw = split ? 2 << (k % 3) : 1 << (si & 3);
        const int pack = (split ? k / 3 : (si >> 2) & 1) ? h->pack_cap : 0;
        const int stage = split ? 0 : budgets[si >> 3];
        h->cfg.warps_per_block = nw;
        h->cfg.pack_agents = pack;
        h->cfg.stage_bytes = stage;
        h->cfg.split_step = split ? 1 : 0;
        e = copy_all(false);
        WorldArgs a = make_args(h);
        a.actions = d_actions;
        a.h = dt / (float)substeps;
        a.substeps = substeps;
        if (e == cudaSuccess) e = launch_step(h, a);   // warm
        if (e == cudaSuccess) e = cudaEventRecord(t0, h->stream);
        for (int it = 0; it < iters && e == cudaSuccess; ++it) e = launch_step(h, a);
        if (e == cudaSuccess) e = cudaEventRecord(t1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[si], t0, t1);
        ms[si] /= (float)iters;
        if (e == cudaSuccess && (first || ms[si] < best_ms)) {
            best_ms = ms[si];
            best = nw;
            best_pack = pack;
            best_stage = stage;
            best_split = split ? 1 : 0;
            first = false;
        }
    }
    if (e == cudaSuccess) e = copy_all(false);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(snap);
    if (e != cudaSuccess) {
        h->cfg.warps_per_block = saved;
        h->cfg.pack_agents = saved_pack;
        h->cfg.stage_bytes = saved_stage;
        h->cfg.split_step = saved_split;
        return cuda_fail(h, e, "sf_autotune");
    }
    h->cfg.warps_per_block = best;
    h->cfg.pack_agents = best_pack;
    h->cfg.stage_bytes = best_stage;
    h->cfg.split_step = best_split;
    if (out_shape) {
        out_shape[0] = best; out_shape[1] = best_pack; out_shape[2] = best_stage; out_shape[3] = best_split;
    }
    if (out_ms) for (int i = 0; i < SF_AUTOTUNE_SHAPES; ++i) out_ms[i] = ms[i];
    return SF_OK;
}

sf_status sf_reset(sf_handle h, const uint8_t* d_mask) {
    if (!h) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_reset: no roads loaded");
    if (!d_mask && h->A > 0) return fail(h, SF_ERR_INVALID_ARG, "sf_reset: mask is NULL");
    WorldArgs a = make_args(h);
    a.mask = d_mask;
    cudaError_t e = sf_launch_world(kModeReset, a, wpb_of(h), h->stream);
    if (e == cudaSuccess && h->m_cnt && h->A > 0) {
        metrics_reset_kernel<<<(h->A + 255) / 256, 256, 0, h->stream>>>(d_mask, h->A, h->m_epmax, h->m_epev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "sf_reset launch");
    return SF_OK;
}

sf_status sf_get_metrics(sf_handle h, sf_metrics* out) {
    if (!h || !out) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_get_metrics: no roads loaded");
    if (!h->m_cnt) return fail(h, SF_ERR_STATE, "sf_get_metrics: the handle was created without SF_FLAG_METRICS");
    unsigned long long c[kMetricCount];
    SF_CUDA(h, cudaMemcpyAsync(c, h->m_cnt, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    SF_CUDA(h, cudaStreamSynchronize(h->stream));
    sf_metrics m{};
    m.episodes = c[kMetricEpisodes];
    m.goals = c[kMetricGoals];
    m.collisions = c[kMetricCollisions];
    m.crashes = c[kMetricCrashes];
    m.offroad = c[kMetricOffroad];
    m.lane_forbidden = c[kMetricLaneForb];
    m.idle = c[kMetricIdle];
    m.timeouts = c[kMetricTimeouts];
    m.nonfinite = c[kMetricNonfinite];
    m.drac_over = c[kMetricDracOver];
    const double n = (double)m.episodes;
    m.success_rate = n > 0 ? (double)m.goals / n : 0.0;
    m.collision_rate = n > 0 ? (double)m.collisions / n : 0.0;
    m.mean_episode_max_drac = n > 0 ? (double)c[kMetricDracMicro] * 1e-6 / n : 0.0;
    m.drac_over_rate = n > 0 ? (double)m.drac_over / n : 0.0;
    *out = m;
    return SF_OK;
}

sf_status sf_reset_metrics(sf_handle h) {
    if (!h) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_reset_metrics: no roads loaded");
    if (!h->m_cnt) return fail(h, SF_ERR_STATE, "sf_reset_metrics: the handle was created without SF_FLAG_METRICS");
    SF_CUDA(h, cudaMemsetAsync(h->m_cnt, 0, kMetricCount * sizeof(unsigned long long), h->stream));
    return SF_OK;
}

sf_status sf_get_obs(sf_handle h, float* d_obs, float* d_reward, uint8_t* d_done, uint32_t* d_events) {
    if (!h) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_get_obs: no roads loaded");
    const size_t A = (size_t)h->A;
    if (d_obs) SF_CUDA(h, cudaMemcpyAsync(d_obs, h->out.obs, A * SF_OBS_DIM * 4, cudaMemcpyDeviceToDevice, h->stream));
    if (d_reward) SF_CUDA(h, cudaMemcpyAsync(d_reward, h->out.reward, A * 4, cudaMemcpyDeviceToDevice, h->stream));
    if (d_done) SF_CUDA(h, cudaMemcpyAsync(d_done, h->out.done, A, cudaMemcpyDeviceToDevice, h->stream));
    if (d_events) SF_CUDA(h, cudaMemcpyAsync(d_events, h->out.events, A * 4, cudaMemcpyDeviceToDevice, h->stream));
    return SF_OK;
}

sf_status sf_get_indices(sf_handle h, int32_t* d_lane_seg, int32_t* d_knn_points, int32_t* d_knn_agents,
                         float* d_drac) {
    if (!h) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_get_indices: no roads loaded");
    const size_t A = (size_t)h->A;
    if (d_lane_seg)
        SF_CUDA(h, cudaMemcpyAsync(d_lane_seg, h->out.lane_seg, A * 4, cudaMemcpyDeviceToDevice, h->stream));
    if (d_knn_points)
        SF_CUDA(h, cudaMemcpyAsync(d_knn_points, h->out.knn_pts, A * SF_L_POINTS * 4, cudaMemcpyDeviceToDevice,
                                   h->stream));
    if (d_knn_agents)
        SF_CUDA(h, cudaMemcpyAsync(d_knn_agents, h->out.knn_agents, A * SF_K_AGENTS * 4, cudaMemcpyDeviceToDevice,
                                   h->stream));
    if (d_drac) SF_CUDA(h, cudaMemcpyAsync(d_drac, h->out.drac, A * 4, cudaMemcpyDeviceToDevice, h->stream));
    return SF_OK;
}

sf_status sf_observe_full(sf_handle h, float* d_obs, int32_t* d_n_road, int32_t* d_n_veh, int32_t* d_road_idx,
                          int32_t* d_veh_idx) {
    if (!h) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_observe_full: no roads loaded");
    if (!d_obs) return fail(h, SF_ERR_INVALID_ARG, "sf_observe_full: NULL observation buffer");
    FullObsArgs f{};
    f.st = h->st;
    f.rd = h->rd;
    f.agent_world = h->sc.agent_world;
    f.num_agents = h->A;
    f.obs = d_obs;
    f.n_road = d_n_road;
    f.n_veh = d_n_veh;
    f.road_idx = d_road_idx;
    f.veh_idx = d_veh_idx;
    f.weather_all = h->cfg.weather_model == SF_WEATHER_ALL ? 1 : 0;
    SF_CUDA(h, sf_launch_full_obs(f, h->stream));
    return SF_OK;
}

sf_status sf_output_ptrs(sf_handle h, sf_outputs* o) {
    if (!h || !o) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_output_ptrs: no roads loaded");
    o->obs = h->out.obs;
    o->reward = h->out.reward;
    o->done = h->out.done;
    o->events = h->out.events;
    o->lane_seg = h->out.lane_seg;
    o->knn_points = h->out.knn_pts;
    o->knn_agents = h->out.knn_agents;
    o->drac = h->out.drac;
    o->num_agents = h->A;
    return SF_OK;
}

static sf_status observe_all(sf_handle h) {
    WorldArgs a = make_args(h);
    cudaError_t e = sf_launch_world(kModeObserve, a, wpb_of(h), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "observe launch");
    return SF_OK;
}

sf_status sf_place_agents(sf_handle h, const float* h_place) {
    if (!h) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_place_agents: no roads loaded");
    if (!h_place && h->A > 0) return fail(h, SF_ERR_INVALID_ARG, "sf_place_agents: NULL");
    for (int i = 0; i < h->A * 6; ++i)
        if (!std::isfinite(h_place[i])) return fail(h, SF_ERR_INVALID_ARG, "sf_place_agents: non-finite value");
    SF_CUDA(h, cudaStreamSynchronize(h->stream));
    SF_CUDA(h, cudaMemcpy(h->place_buf, h_place, (size_t)h->A * 6 * 4, cudaMemcpyHostToDevice));
    WorldArgs a = make_args(h);
    cudaError_t e = sf_launch_place(a, h->place_buf, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "place launch");
    sf_status s = observe_all(h);
    if (s != SF_OK) return s;
    SF_CUDA(h, cudaStreamSynchronize(h->stream));
    return SF_OK;
}

sf_status sf_get_state(sf_handle h, float* h_f, int32_t* h_i) {
    if (!h) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_get_state: no roads loaded");
    if ((!h_f || !h_i) && h->A > 0) return fail(h, SF_ERR_INVALID_ARG, "sf_get_state: NULL");
    SF_CUDA(h, cudaStreamSynchronize(h->stream));
    const size_t A = (size_t)h->A;
    std::vector<float4> pos(A), quat(A), vel(A), angv(A), spin(A), goal(A);
    std::vector<float> peak(A);
    std::vector<uint32_t> meta(A), events(A);
    std::vector<int32_t> step(A), episode(A);
    if (A) {
        SF_CUDA(h, cudaMemcpy(pos.data(), h->st.pos, A * 16, cudaMemcpyDeviceToHost));
        SF_CUDA(h, cudaMemcpy(quat.data(), h->st.quat, A * 16, cudaMemcpyDeviceToHost));
        SF_CUDA(h, cudaMemcpy(vel.data(), h->st.vel, A * 16, cudaMemcpyDeviceToHost));
        SF_CUDA(h, cudaMemcpy(angv.data(), h->st.angv, A * 16, cudaMemcpyDeviceToHost));
        SF_CUDA(h, cudaMemcpy(spin.data(), h->st.spin, A * 16, cudaMemcpyDeviceToHost));
        SF_CUDA(h, cudaMemcpy(goal.data(), h->st.goal, A * 16, cudaMemcpyDeviceToHost));
        SF_CUDA(h, cudaMemcpy(peak.data(), h->st.peak_drac, A * 4, cudaMemcpyDeviceToHost));
        SF_CUDA(h, cudaMemcpy(meta.data(), h->st.meta, A * 4, cudaMemcpyDeviceToHost));
        SF_CUDA(h, cudaMemcpy(step.data(), h->st.step, A * 4, cudaMemcpyDeviceToHost));
        SF_CUDA(h, cudaMemcpy(episode.data(), h->st.episode, A * 4, cudaMemcpyDeviceToHost));
        SF_CUDA(h, cudaMemcpy(events.data(), h->out.events, A * 4, cudaMemcpyDeviceToHost));
    }
    for (size_t a = 0; a < A; ++a) {
        float* f = h_f + a * SF_NF;
        f[SF_F_PX] = pos[a].x; f[SF_F_PY] = pos[a].y; f[SF_F_PZ] = pos[a].z; f[SF_F_DELTA] = pos[a].w;
        f[SF_F_QW] = quat[a].x; f[SF_F_QX] = quat[a].y; f[SF_F_QY] = quat[a].z; f[SF_F_QZ] = quat[a].w;
        f[SF_F_VX] = vel[a].x; f[SF_F_VY] = vel[a].y; f[SF_F_VZ] = vel[a].z; f[SF_F_DDELTA] = vel[a].w;
        f[SF_F_WX] = angv[a].x; f[SF_F_WY] = angv[a].y; f[SF_F_WZ] = angv[a].z; f[SF_F_MU] = angv[a].w;
        f[SF_F_S0] = spin[a].x; f[SF_F_S1] = spin[a].y; f[SF_F_S2] = spin[a].z; f[SF_F_S3] = spin[a].w;
        f[SF_F_GX] = goal[a].x; f[SF_F_GY] = goal[a].y; f[SF_F_SX] = goal[a].z; f[SF_F_SY] = goal[a].w;
        f[SF_F_PEAK_DRAC] = peak[a];
        int32_t* i = h_i + a * SF_NI;
        i[SF_I_PRECIP] = (int32_t)(meta[a] & 0xFF);
        i[SF_I_SURFACE] = (int32_t)((meta[a] >> 8) & 0xFF);
        i[SF_I_STATUS] = (int32_t)((meta[a] >> 16) & 0xFF);
        i[SF_I_STEP] = step[a];
        i[SF_I_EPISODE] = episode[a];
        i[SF_I_EVENTS] = (int32_t)events[a];
    }
    return sf_sync(h);
}

sf_status sf_set_state(sf_handle h, const float* h_f, const int32_t* h_i) {
    if (!h) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_set_state: no roads loaded");
    if ((!h_f || !h_i) && h->A > 0) return fail(h, SF_ERR_INVALID_ARG, "sf_set_state: NULL");
    const size_t A = (size_t)h->A;
    for (size_t a = 0; a < A; ++a) {
        const int32_t* i = h_i + a * SF_NI;
        if (i[SF_I_PRECIP] < 0 || i[SF_I_PRECIP] > 3 || i[SF_I_SURFACE] < 0 || i[SF_I_SURFACE] > 2 ||
            i[SF_I_STATUS] < 0 || i[SF_I_STATUS] > 3)
            return fail(h, SF_ERR_INVALID_ARG, "sf_set_state: bad int state at agent " + std::to_string(a));
    }
    std::vector<float4> pos(A), quat(A), vel(A), angv(A), spin(A), goal(A);
    std::vector<float> peak(A);
    std::vector<uint32_t> meta(A), events(A);
    std::vector<int32_t> step(A), episode(A);
    for (size_t a = 0; a < A; ++a) {
        const float* f = h_f + a * SF_NF;
        pos[a] = make_float4(f[SF_F_PX], f[SF_F_PY], f[SF_F_PZ], f[SF_F_DELTA]);
        quat[a] = make_float4(f[SF_F_QW], f[SF_F_QX], f[SF_F_QY], f[SF_F_QZ]);
        vel[a] = make_float4(f[SF_F_VX], f[SF_F_VY], f[SF_F_VZ], f[SF_F_DDELTA]);
        angv[a] = make_float4(f[SF_F_WX], f[SF_F_WY], f[SF_F_WZ], f[SF_F_MU]);
        spin[a] = make_float4(f[SF_F_S0], f[SF_F_S1], f[SF_F_S2], f[SF_F_S3]);
        goal[a] = make_float4(f[SF_F_GX], f[SF_F_GY], f[SF_F_SX], f[SF_F_SY]);
        peak[a] = f[SF_F_PEAK_DRAC];
        const int32_t* i = h_i + a * SF_NI;
        meta[a] = (uint32_t)i[SF_I_PRECIP] | ((uint32_t)i[SF_I_SURFACE] << 8) | ((uint32_t)i[SF_I_STATUS] << 16);
        step[a] = i[SF_I_STEP];
        episode[a] = i[SF_I_EPISODE];
        events[a] = (uint32_t)i[SF_I_EVENTS];
    }
    SF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (A) {
        SF_CUDA(h, cudaMemcpy(h->st.pos, pos.data(), A * 16, cudaMemcpyHostToDevice));
        SF_CUDA(h, cudaMemcpy(h->st.quat, quat.data(), A * 16, cudaMemcpyHostToDevice));
        SF_CUDA(h, cudaMemcpy(h->st.vel, vel.data(), A * 16, cudaMemcpyHostToDevice));
        SF_CUDA(h, cudaMemcpy(h->st.angv, angv.data(), A * 16, cudaMemcpyHostToDevice));
        SF_CUDA(h, cudaMemcpy(h->st.spin, spin.data(), A * 16, cudaMemcpyHostToDevice));
        SF_CUDA(h, cudaMemcpy(h->st.goal, goal.data(), A * 16, cudaMemcpyHostToDevice));
        SF_CUDA(h, cudaMemcpy(h->st.peak_drac, peak.data(), A * 4, cudaMemcpyHostToDevice));
        SF_CUDA(h, cudaMemcpy(h->st.meta, meta.data(), A * 4, cudaMemcpyHostToDevice));
        SF_CUDA(h, cudaMemcpy(h->st.step, step.data(), A * 4, cudaMemcpyHostToDevice));
        SF_CUDA(h, cudaMemcpy(h->st.episode, episode.data(), A * 4, cudaMemcpyHostToDevice));
        SF_CUDA(h, cudaMemcpy(h->out.events, events.data(), A * 4, cudaMemcpyHostToDevice));
    }
    sf_status s = observe_all(h);
    if (s != SF_OK) return s;
    SF_CUDA(h, cudaStreamSynchronize(h->stream));
    return SF_OK;
}

static const char kMagic[8] = {'S', 'F', 'C', 'K', 'P', 'T', '0', '1'};

sf_status sf_save_state(sf_handle h, const char* path) {
    if (!h || !path) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_save_state: no roads loaded");
    std::vector<float> f((size_t)h->A * SF_NF);
    std::vector<int32_t> i((size_t)h->A * SF_NI);
    sf_status s = sf_get_state(h, f.data(), i.data());
    if (s != SF_OK && s != SF_ERR_NONFINITE) return s;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(h, SF_ERR_INVALID_ARG, std::string("sf_save_state: cannot open ") + path);
    int32_t hdr[4] = {h->A, SF_NF, SF_NI, h->W};
    bool ok = std::fwrite(kMagic, 1, 8, fp) == 8 && std::fwrite(hdr, 4, 4, fp) == 4 &&
              std::fwrite(f.data(), 4, f.size(), fp) == f.size() && std::fwrite(i.data(), 4, i.size(), fp) == i.size();
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? s : fail(h, SF_ERR_INVALID_ARG, "sf_save_state: write failed");
}

sf_status sf_load_state(sf_handle h, const char* path) {
    if (!h || !path) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_load_state: no roads loaded");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(h, SF_ERR_INVALID_ARG, std::string("sf_load_state: cannot open ") + path);
    char magic[8];
    int32_t hdr[4];
    bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, kMagic, 8) == 0 && std::fread(hdr, 4, 4, fp) == 4 &&
              hdr[0] == h->A && hdr[1] == SF_NF && hdr[2] == SF_NI && hdr[3] == h->W;
    std::vector<float> f((size_t)h->A * SF_NF);
    std::vector<int32_t> i((size_t)h->A * SF_NI);
    ok = ok && std::fread(f.data(), 4, f.size(), fp) == f.size() && std::fread(i.data(), 4, i.size(), fp) == i.size();
    std::fclose(fp);
    if (!ok) return fail(h, SF_ERR_INVALID_ARG, "sf_load_state: bad or mismatched checkpoint");
    return sf_set_state(h, f.data(), i.data());
}

sf_status sf_step_policy(sf_handle h, sf_mlp_handle policy, float dt, int substeps) {
    if (!h || !policy) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_step_policy: no roads loaded");
    sf_status s = sf_mlp_forward_on(policy, h->stream, h->out.obs, SF_OBS_DIM, h->A, h->act_buf, 3);
    if (s != SF_OK) return fail(h, s, std::string("sf_step_policy: ") + sf_mlp_last_error(policy));
    return sf_step(h, h->act_buf, dt, substeps);
}

// observe (full), act (late-fusion actor mean, critic value), step
static sf_status lf_step_body(sf_handle h, sf_lf_handle lf, LfBufs* b, float dt, int substeps) {
    sf_status s = sf_observe_full(h, b->obs, b->n_road, b->n_veh, nullptr, nullptr);
    if (s != SF_OK) return s;
    s = sf_lf_forward_on(lf, h->stream, b->obs, b->n_road, b->n_veh, h->A, h->act_buf, b->value, nullptr);
    if (s != SF_OK) return fail(h, s, std::string("late-fusion forward: ") + sf_lf_last_error(lf));
    return sf_step(h, h->act_buf, dt, substeps);
}

sf_status sf_step_lf(sf_handle h, sf_lf_handle lf, float dt, int substeps) {
    if (!h || !lf) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_step_lf: no roads loaded");
    LfBufs* b = lf_bufs(h);
    if (!b) return fail(h, SF_ERR_OOM, "sf_step_lf: observation buffers");
    return lf_step_body(h, lf, b, dt, substeps);
}

sf_status sf_lf_step_outputs(sf_handle h, sf_lf_outputs* o) {
    if (!h || !o) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_lf_step_outputs: no roads loaded");
    LfBufs* b = lf_bufs(h);
    if (!b) return fail(h, SF_ERR_OOM, "sf_lf_step_outputs: observation buffers");
    o->obs = b->obs;
    o->n_road = b->n_road;
    o->n_veh = b->n_veh;
    o->actions = h->act_buf;
    o->value = b->value;
    o->num_agents = h->A;
    return SF_OK;
}

sf_status sf_graph_capture_lf(sf_handle h, sf_lf_handle lf, const uint8_t* d_reset_mask, float dt, int substeps,
                              sf_graph_handle* out) {
    if (!h || !lf || !out) return SF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_graph_capture_lf: no roads loaded");
    if (!h->stream) return fail(h, SF_ERR_INVALID_ARG, "sf_graph_capture_lf: needs a non-default stream");
    LfBufs* b = lf_bufs(h);
    if (!b || sf_lf_reserve(lf, h->A) != SF_OK) return fail(h, SF_ERR_OOM, "sf_graph_capture_lf: buffers");
    // one uncaptured forward: first-use work (kernel attributes) happens outside the capture
    sf_status s0 = sf_observe_full(h, b->obs, b->n_road, b->n_veh, nullptr, nullptr);
    if (s0 == SF_OK) s0 = sf_lf_forward_on(lf, h->stream, b->obs, b->n_road, b->n_veh, h->A, h->act_buf, b->value, nullptr);
    if (s0 != SF_OK) return fail(h, s0, "sf_graph_capture_lf: warm-up forward");
    SF_CUDA(h, cudaStreamSynchronize(h->stream));
    sf_graph* g = new sf_graph();
    g->h = h;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    sf_status st = SF_OK;
    if (e == cudaSuccess) {
        st = lf_step_body(h, lf, b, dt, substeps);
        g->launches = 16;
        if (st == SF_OK && d_reset_mask) { st = sf_reset(h, d_reset_mask); g->launches += 1; }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
        if (e2 == cudaSuccess && st == SF_OK) {
            g->graph = graph;
            e = cudaGraphInstantiate(&g->exec, graph, 0);
        } else {
            if (graph) cudaGraphDestroy(graph);
            e = e2 != cudaSuccess ? e2 : cudaErrorUnknown;
        }
    }
    if (e != cudaSuccess || st != SF_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return st != SF_OK ? st : cuda_fail(h, e, "sf_graph_capture_lf");
    }
    *out = g;
    return SF_OK;
}

sf_status sf_graph_capture(sf_handle h, sf_mlp_handle policy, sf_surrogate_handle surrogate, const float* d_actions,
                           const uint8_t* d_reset_mask, float dt, int substeps, sf_graph_handle* out) {
    if (!h || !out) return SF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_graph_capture: no roads loaded");
    if (!policy && !d_actions) return fail(h, SF_ERR_INVALID_ARG, "sf_graph_capture: no actions and no policy");
    if (!h->stream) return fail(h, SF_ERR_INVALID_ARG, "sf_graph_capture: needs a non-default stream");
    if (policy && sf_mlp_reserve(policy, h->A) != SF_OK)
        return fail(h, SF_ERR_OOM, "sf_graph_capture: policy buffers");
    if (policy) {   // one uncaptured pass: first-use work (kernel attributes) happens outside the capture
        sf_status s0 = sf_mlp_forward_on(policy, h->stream, h->out.obs, SF_OBS_DIM, h->A, h->act_buf, 3);
        if (s0 != SF_OK) return fail(h, s0, "sf_graph_capture: policy forward");
    }
    if (surrogate) {
        SurrBufs* b = surr_bufs(h);
        if (!b || sf_mlp_reserve(surrogate->mlp, h->A) != SF_OK)
            return fail(h, SF_ERR_OOM, "sf_graph_capture: surrogate buffers");
        sf_status s0 = sf_mlp_forward_on(surrogate->mlp, h->stream, b->x, kSurrInLd, h->A, b->y, kSurrOut);
        if (s0 != SF_OK) return fail(h, s0, "sf_graph_capture: surrogate forward");
    }
    SF_CUDA(h, cudaStreamSynchronize(h->stream));
    sf_graph* g = new sf_graph();
    g->h = h;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    sf_status st = SF_OK;
    if (e == cudaSuccess) {
        if (policy) {
            st = sf_mlp_forward_on(policy, h->stream, h->out.obs, SF_OBS_DIM, h->A, h->act_buf, 3);
            g->launches += 1;
        }
        const float* acts = policy ? h->act_buf : d_actions;
        if (st == SF_OK) {
            if (surrogate) { st = sf_step_surrogate(h, surrogate, acts, dt, substeps, 0); g->launches += 5; }
            else { st = sf_step(h, acts, dt, substeps); g->launches += 1; }
        }
        if (st == SF_OK && d_reset_mask) { st = sf_reset(h, d_reset_mask); g->launches += 1; }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
        if (e2 == cudaSuccess && st == SF_OK) {
            g->graph = graph;
            e = cudaGraphInstantiate(&g->exec, graph, 0);
        } else {
            if (graph) cudaGraphDestroy(graph);
            e = e2 != cudaSuccess ? e2 : cudaErrorUnknown;
        }
    }
    if (e != cudaSuccess || st != SF_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return st != SF_OK ? st : cuda_fail(h, e, "sf_graph_capture");
    }
    *out = g;
    return SF_OK;
}

sf_status sf_graph_launch(sf_graph_handle g) {
    if (!g) return SF_ERR_INVALID_ARG;
    cudaError_t e = cudaGraphLaunch(g->exec, g->h->stream);
    return e == cudaSuccess ? SF_OK : cuda_fail(g->h, e, "sf_graph_launch");
}

sf_status sf_graph_destroy(sf_graph_handle g) {
    if (!g) return SF_OK;
    cudaStreamSynchronize(g->h->stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return SF_OK;
}

// ====================================================================== dynamics surrogate

sf_status sf_surrogate_create(void* cuda_stream, sf_surrogate_handle* out) {
    if (!out) return SF_ERR_INVALID_ARG;
    *out = nullptr;
    sf_surrogate* s = new sf_surrogate();
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    const int32_t dims[5] = {kSurrIn, 256, 256, 256, kSurrOut};
    sf_status st = sf_mlp_create(4, dims, SF_ACT_SILU, SF_ACT_NONE, cuda_stream, &s->mlp);
    if (st != SF_OK) { delete s; return st; }
    cudaError_t e = cudaMalloc(&s->stats, 2 * (kSurrIn + kSurrOut) * sizeof(float));
    if (e != cudaSuccess) { sf_mlp_destroy(s->mlp); delete s; return SF_ERR_OOM; }
    // identity statistics until trained
    std::vector<float> st0(2 * (kSurrIn + kSurrOut), 0.f);
    for (int i = 0; i < kSurrIn; ++i) st0[kSurrIn + i] = 1.f;
    for (int i = 0; i < kSurrOut; ++i) st0[2 * kSurrIn + kSurrOut + i] = 1.f;
    cudaMemcpy(s->stats, st0.data(), st0.size() * 4, cudaMemcpyHostToDevice);
    // He-style initialisation with a fixed seed (weights are trained afterwards)
    uint64_t z = 0x5EEDull;
    auto rnd = [&]() {
        z += 0x9E3779B97F4A7C15ull;
        uint64_t q = z;
        q = (q ^ (q >> 30)) * 0xBF58476D1CE4E5B9ull;
        q = (q ^ (q >> 27)) * 0x94D049BB133111EBull;
        q ^= q >> 31;
        return ((double)(q >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
    };
    for (int l = 0; l < 4; ++l) {
        const int i = dims[l], o = dims[l + 1];
        std::vector<float> w((size_t)o * i), b((size_t)o, 0.f);
        const double a = std::sqrt(6.0 / i) * (l == 3 ? 0.1 : 1.0);
        for (auto& v : w) v = (float)(a * rnd());
        st = sf_mlp_set_layer(s->mlp, l, w.data(), b.data());
        if (st != SF_OK) break;
    }
    if (st != SF_OK) { sf_surrogate_destroy(s); return st; }
    *out = s;
    return SF_OK;
}

sf_status sf_surrogate_destroy(sf_surrogate_handle s) {
    if (!s) return SF_OK;
    if (s->mlp) sf_mlp_destroy(s->mlp);
    cudaFree(s->stats);
    cudaFree(s->bx);
    cudaFree(s->by);
    delete s;
    return SF_OK;
}

sf_status sf_surrogate_collect(sf_handle h, sf_surrogate_handle s, const float* d_actions, float dt, int substeps,
                               float* d_x, float* d_y, unsigned long long cap, unsigned long long* d_count) {
    if (!h || !s || !d_actions || !d_x || !d_y || !d_count) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_surrogate_collect: no roads loaded");
    if (h->cfg.dynamics != SF_DYN_VEHICLE)
        return fail(h, SF_ERR_STATE, "sf_surrogate_collect: the surrogate learns the raycast vehicle only");
    SurrBufs* b = surr_bufs(h);
    if (!b) return fail(h, SF_ERR_OOM, "sf_surrogate_collect: buffers");
    WorldArgs a = make_args(h);
    cudaError_t e = sf_launch_surr_gate(a, dt, b->elig, h->stream);
    if (e == cudaSuccess) e = sf_launch_surr_features(a, d_actions, nullptr, b->x, h->stream);
    if (e == cudaSuccess) e = sf_launch_surr_snapshot(a, b->snap, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "sf_surrogate_collect");
    sf_status st = sf_step(h, d_actions, dt, substeps);
    if (st != SF_OK) return st;
    e = sf_launch_surr_collect(a, b->snap, b->elig, b->x, dt, d_x, d_y, cap, d_count, h->stream);
    return e == cudaSuccess ? SF_OK : cuda_fail(h, e, "sf_surrogate_collect");
}

sf_status sf_surrogate_train(sf_surrogate_handle s, const float* d_x, const float* d_y, unsigned long long n,
                             int batch, int steps, float lr, unsigned long long seed, float* h_loss) {
    if (!s || !d_x || !d_y || n == 0 || batch < 8 || batch % 8 || steps < 0) return SF_ERR_INVALID_ARG;
    cudaError_t e = cudaSuccess;
    if (batch > s->bcap) {
        cudaFree(s->bx);
        cudaFree(s->by);
        s->bx = s->by = nullptr;
        e = cudaMalloc(&s->bx, (size_t)batch * kSurrIn * 4);
        if (e == cudaSuccess) e = cudaMalloc(&s->by, (size_t)batch * kSurrOut * 4);
        if (e != cudaSuccess) { s->err = "sf_surrogate_train: buffers"; return SF_ERR_OOM; }
        s->bcap = batch;
    }
    e = sf_launch_col_stats(d_x, n, kSurrIn, s->stats, s->stream);
    if (e == cudaSuccess) e = sf_launch_col_stats(d_y, n, kSurrOut, s->stats + 2 * kSurrIn, s->stream);
    if (e != cudaSuccess) { s->err = cudaGetErrorString(e); return SF_ERR_CUDA; }
    float loss = 0.f;
    for (int t = 0; t < steps; ++t) {
        // cosine decay to 5% of the initial rate
        const float lr_t = lr * (0.05f + 0.95f * 0.5f * (1.f + std::cos(3.14159265f * (float)t / (float)steps)));
        e = sf_launch_gather(d_x, d_y, n, s->stats, s->stats + 2 * kSurrIn, batch, seed, (unsigned long long)t, s->bx,
                             s->by, s->stream);
        if (e != cudaSuccess) { s->err = cudaGetErrorString(e); return SF_ERR_CUDA; }
        const bool last = t == steps - 1;
        sf_status st = sf_mlp_train_step(s->mlp, s->bx, s->by, batch, lr_t, 1, (last && h_loss) ? &loss : nullptr);
        if (st != SF_OK) { s->err = sf_mlp_last_error(s->mlp); return st; }
    }
    if (h_loss) *h_loss = loss;
    s->trained = true;
    return sf_mlp_sync(s->mlp);
}

sf_mlp_handle sf_surrogate_mlp(sf_surrogate_handle s) { return s ? s->mlp : nullptr; }

sf_status sf_surrogate_stats(sf_surrogate_handle s, float* h_stats) {
    if (!s || !h_stats) return SF_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaMemcpy(h_stats, s->stats, 2 * (kSurrIn + kSurrOut) * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SF_OK : SF_ERR_CUDA;
}

sf_status sf_surrogate_set_stats(sf_surrogate_handle s, const float* h_stats) {
    if (!s || !h_stats) return SF_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaMemcpy(s->stats, h_stats, 2 * (kSurrIn + kSurrOut) * 4, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? SF_OK : SF_ERR_CUDA;
}

sf_status sf_step_surrogate(sf_handle h, sf_surrogate_handle s, const float* d_actions, float dt, int substeps,
                            int audit) {
    if (!h || !s || !d_actions) return SF_ERR_INVALID_ARG;
    if (!h->loaded) return fail(h, SF_ERR_STATE, "sf_step_surrogate: no roads loaded");
    if (h->cfg.dynamics != SF_DYN_VEHICLE)
        return fail(h, SF_ERR_STATE, "sf_step_surrogate: the surrogate replaces the raycast vehicle only");
    if (!(dt > 0.f) || substeps < 1 || substeps > 64) return fail(h, SF_ERR_INVALID_ARG, "sf_step_surrogate: dt");
    SurrBufs* b = surr_bufs(h);
    if (!b) return fail(h, SF_ERR_OOM, "sf_step_surrogate: buffers");
    WorldArgs a = make_args(h);
    cudaError_t e = sf_launch_surr_features(a, d_actions, s->stats, b->x, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "sf_step_surrogate features");
    sf_status st = sf_mlp_forward_on(s->mlp, h->stream, b->x, kSurrInLd, h->A, b->y, kSurrOut);
    if (st != SF_OK) return fail(h, st, std::string("sf_step_surrogate: ") + sf_mlp_last_error(s->mlp));
    a.actions = d_actions;
    a.h = dt / (float)substeps;
    a.substeps = substeps;
    a.surr_y = b->y;
    a.surr_stats = s->stats + 2 * kSurrIn;
    a.surr_mode = audit ? 2 : 1;
    a.audit_err = b->words;
    a.surr_count = b->words + 1;
    e = launch_step(h, a);
    if (e == cudaSuccess) e = launch_metrics(h);
    return e == cudaSuccess ? SF_OK : cuda_fail(h, e, "sf_step_surrogate");
}

sf_status sf_surrogate_audit(sf_handle h, float* h_max_err, unsigned long long* h_used) {
    if (!h) return SF_ERR_INVALID_ARG;
    SurrBufs* b = surr_bufs(h);
    if (!b) return fail(h, SF_ERR_OOM, "sf_surrogate_audit: buffers");
    unsigned w[2] = {0, 0};
    SF_CUDA(h, cudaStreamSynchronize(h->stream));
    SF_CUDA(h, cudaMemcpy(w, b->words, 8, cudaMemcpyDeviceToHost));
    SF_CUDA(h, cudaMemset(b->words, 0, 8));
    float f;
    std::memcpy(&f, &w[0], 4);
    if (h_max_err) *h_max_err = f;
    if (h_used) *h_used = w[1];
    return SF_OK;
}

sf_status sf_set_wait_limit(sf_handle h, unsigned long long limit_ns, int withhold_producer) {
    if (!h) return SF_ERR_INVALID_ARG;
    h->wait_ns = limit_ns == 0 ? 1ull : limit_ns;   // the kernels read 0 as the 1 s default
    h->withhold = withhold_producer != 0;
    return SF_OK;
}

sf_status sf_sync(sf_handle h) {
    if (!h) return SF_ERR_INVALID_ARG;
    SF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (!h->loaded) return SF_OK;
    unsigned int w = 0;
    SF_CUDA(h, cudaMemcpy(&w, h->out.error_word, 4, cudaMemcpyDeviceToHost));
    if (w) {
        SF_CUDA(h, cudaMemset(h->out.error_word, 0, 4));
        if (w & 1u) return fail(h, SF_ERR_NONFINITE, "an agent state went non-finite (agent parked or respawned)");
        return fail(h, SF_ERR_TIMEOUT, "a bounded device wait gave up");
    }
    return SF_OK;
}

}  // extern "C"

