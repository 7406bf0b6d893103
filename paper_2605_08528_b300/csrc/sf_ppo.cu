// sf_ppo.cu -- on-device PPO (SceneFactory App. L, Tab. app_ppo_hparams; the
// training loop of Alg. 1) with the BF16 tensor-core MLPs of sf_mlp.cu.
//
// The policy is a diagonal Gaussian: mean = the actor MLP's output on the
// step's observation, log standard deviation = a free 3-vector.  A rollout of
// `horizon` control steps records, per step and agent, the observation, the
// sampled action (mean + sigma * N(0, 1) from a counter-hashed Box-Muller
// draw), its log-probability, the mean, the critic's value, and the step's
// reward and done flag.  The update computes GAE advantages and returns,
// normalises the advantages over the rollout and runs `epochs` passes of
// `minibatches` minibatches: gather the rows, forward both MLPs keeping their
// activations, the clipped-surrogate / value / entropy loss gradients and the
// Gaussian KL to the rollout policy, backward both MLPs, the learning rate
// adapted on the device from the KL (halved above twice the target, doubled
// below half of it), the global gradient norm clipped, and Adam.  Nothing of
// the update returns to the host until its statistics are read.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/sf.h"
#include "sf_internal.cuh"
#include "sf_mlp_internal.cuh"

namespace {

constexpr int kObsW = SF_OBS_DIM;   // 320
constexpr float kHalfLog2Pi = 0.91893853320467274f;
constexpr float kLrMin = 1e-6f, kLrMax = 1e-2f;

// scalar slots in device memory
enum {
    S_LR = 0,        // current learning rate
    S_SCALE,         // gradient scale of the minibatch (norm clipping)
    S_SUMSQ,         // sum of squared gradients of the minibatch
    S_POL, S_VAL, S_KL,   // minibatch sums: policy loss, value loss, KL
    S_ACC_POL, S_ACC_VAL, S_ACC_KL, S_ACC_NORM,   // sums over the update's minibatches
    S_REW,           // rollout reward sum
    S_COUNT = 16
};

__device__ __forceinline__ unsigned long long smix(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
// uniform in (0, 1]: the top 24 bits of a hash, plus one, over 2^24
__device__ __forceinline__ float u24p(unsigned long long h) {
    return ((float)(uint32_t)(h >> 40) + 1.f) * (1.f / 16777216.f);
}

__device__ __forceinline__ float logp3(const float* a, const float* mu, const float* s) {
    float lp = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float d = a[i] - mu[i];
        lp += -d * d / (2.f * __expf(2.f * s[i])) - s[i] - kHalfLog2Pi;
    }
    return lp;
}

// actions and their log-probabilities for one rollout step
__global__ void sample_kernel(const float* __restrict__ mu, const float* __restrict__ log_std, int A,
                              unsigned long long seed, unsigned long long step, float* __restrict__ act,
                              float* __restrict__ logp) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A) return;
    const unsigned long long key = seed ^ smix((step * 0x100000001B3ull) ^ (unsigned long long)a);
    float z[4];
#pragma unroll
    for (int k = 0; k < 2; ++k) {   // Box-Muller: two normals from two uniforms
        const float u1 = u24p(smix(key + 4 * k)), u2 = u24p(smix(key + 4 * k + 1));
        const float r = sqrtf(-2.f * __logf(u1));
        float sn, cs;
        __sincosf(6.283185307179586f * u2, &sn, &cs);
        z[2 * k] = r * cs;
        z[2 * k + 1] = r * sn;
    }
    float s[3], m[3], x[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        s[i] = log_std[i];
        m[i] = mu[3 * (size_t)a + i];
        x[i] = m[i] + __expf(s[i]) * z[i];
        act[3 * (size_t)a + i] = x[i];
    }
    logp[a] = logp3(x, m, s);
}

// rewards [T][A] and done flags, one step at a time
__global__ void record_step_kernel(const float* __restrict__ rew_in, const uint8_t* __restrict__ done_in, int A,
                                   float* __restrict__ rew, uint8_t* __restrict__ done) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < A) {
        rew[a] = rew_in[a];
        done[a] = done_in[a];
    }
}

// Deterministic sums: every reduction of the update adds per-block partial
// sums (warps and then the block's warps in a fixed order) and then the
// partials in order on one thread, so repeated runs agree bit for bit.
template <int K, class T>
__device__ __forceinline__ void block_sums(T (&v)[K], T* out) {   // 256 threads; out[K] on thread 0
    __shared__ T red[8][K];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xFFFFFFFFu, v[k], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[threadIdx.x >> 5][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            T t = 0;
            for (int w = 0; w < 8; ++w) t += red[w][k];
            out[k] = t;
        }
}

// sum of n values: block j sums the j-th of gridDim.x contiguous chunks
constexpr int kSumBlocks = 148;
__global__ void sum_part_kernel(const float* __restrict__ x, size_t n, float* __restrict__ part) {
    const size_t chunk = (n + gridDim.x - 1) / gridDim.x, i0 = (size_t)blockIdx.x * chunk;
    const size_t i1 = i0 + chunk < n ? i0 + chunk : n;
    float v[1] = {0.f};
    for (size_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) v[0] += x[i];
    block_sums<1>(v, part + blockIdx.x);
}
// out[k] (op) sum over j of part[j * stride + k], k < K, in order of j
template <class T>
__global__ void parts_final_kernel(const T* __restrict__ part, int P, int stride, int K, T* __restrict__ out,
                                   bool accumulate) {
    const int k = threadIdx.x;
    if (k >= K) return;
    T t = 0;
    for (int j = 0; j < P; ++j) t += part[(size_t)j * stride + k];
    out[k] = accumulate ? out[k] + t : t;
}

// GAE per agent (one thread): delta_t = r_t + g (1 - d_t) V_{t+1} - V_t, A_t = delta_t + g l (1 - d_t) A_{t+1}
__global__ void gae_kernel(const float* __restrict__ rew, const uint8_t* __restrict__ done,
                           const float* __restrict__ val, int T, int A, float gamma, float lam,
                           float* __restrict__ adv, float* __restrict__ ret, double* __restrict__ mpart) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    double s1 = 0.0, s2 = 0.0;
    if (a < A) {
        float nv = val[(size_t)T * A + a], na = 0.f;
        for (int t = T - 1; t >= 0; --t) {
            const size_t i = (size_t)t * A + a;
            const float keep = done[i] ? 0.f : 1.f;
            const float v = val[i];
            const float delta = rew[i] + gamma * keep * nv - v;
            na = delta + gamma * lam * keep * na;
            adv[i] = na;
            ret[i] = na + v;
            nv = v;
            s1 += na;
            s2 += (double)na * na;
        }
    }
    double v[2] = {s1, s2};
    block_sums<2>(v, mpart + 2 * (size_t)blockIdx.x);   // summed in order into the moments
}

// advantages -> (A - mean) / (std + 1e-8) over the rollout (population std)
__global__ void normalise_kernel(float* __restrict__ adv, size_t n, const double* __restrict__ moments) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double mean = moments[0] / (double)n;
    const double var = fmax(moments[1] / (double)n - mean * mean, 0.0);
    adv[i] = (float)((adv[i] - mean) / (sqrt(var) + 1e-8));
}

// one minibatch: rows (a_e i + b_e) mod N for i in [i0, i0 + B)
struct Perm {
    unsigned long long mul, add, n;
};
__device__ __forceinline__ size_t perm_row(const Perm& p, size_t i) { return (size_t)((p.mul * i + p.add) % p.n); }

__global__ void gather_kernel(Perm p, size_t i0, int B, int W, const float* __restrict__ obs,
                              const float* __restrict__ act, const float* __restrict__ mu,
                              const float* __restrict__ logp, const float* __restrict__ adv,
                              const float* __restrict__ ret, float* __restrict__ g_obs, float* __restrict__ g_small,
                              const int32_t* __restrict__ nr, const int32_t* __restrict__ nv, int32_t* __restrict__ g_nr,
                              int32_t* __restrict__ g_nv) {
    // one warp per row: the W-float observation (coalesced float4 copies when W % 4 == 0),
    // the group counts of a full observation, then the small fields
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= B) return;
    const size_t r = perm_row(p, i0 + row);
    if (W % 4 == 0) {
        const float4* src = reinterpret_cast<const float4*>(obs + r * W);
        float4* dst = reinterpret_cast<float4*>(g_obs + (size_t)row * W);
        for (int k = lane; k < W / 4; k += 32) dst[k] = src[k];
    } else {
        for (int k = lane; k < W; k += 32) g_obs[(size_t)row * W + k] = obs[r * W + k];
    }
    if (nr && lane == 6) g_nr[row] = nr[r];
    if (nv && lane == 7) g_nv[row] = nv[r];
    if (lane < 3) {
        g_small[(size_t)row * 12 + lane] = act[3 * r + lane];
        g_small[(size_t)row * 12 + 3 + lane] = mu[3 * r + lane];
    }
    if (lane == 3) g_small[(size_t)row * 12 + 6] = logp[r];
    if (lane == 4) g_small[(size_t)row * 12 + 7] = adv[r];
    if (lane == 5) g_small[(size_t)row * 12 + 8] = ret[r];
}

// loss gradients of a minibatch row (one thread per row) and block sums of the
// log-std gradient, losses and KL
__global__ void loss_grad_kernel(int B, const float* __restrict__ g_small, const float* __restrict__ mu_new,
                                 const float* __restrict__ v_new, const float* __restrict__ log_std,
                                 const float* __restrict__ log_std_old, float clip, float vf_coef,
                                 float* __restrict__ d_mu, float* __restrict__ d_v, float* __restrict__ lpart) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    float ds[3] = {0.f, 0.f, 0.f}, pol = 0.f, vl = 0.f, kl = 0.f;
    if (row < B) {
        const float* g = g_small + (size_t)row * 12;
        float a[3], mo[3], mn[3], s[3], so[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            a[i] = g[i]; mo[i] = g[3 + i]; mn[i] = mu_new[3 * (size_t)row + i];
            s[i] = log_std[i]; so[i] = log_std_old[i];
        }
        const float lpo = g[6], adv = g[7], ret = g[8];
        const float ratio = __expf(logp3(a, mn, s) - lpo);
        const float unc = ratio * adv, cl = fminf(fmaxf(ratio, 1.f - clip), 1.f + clip) * adv;
        pol = -fminf(unc, cl);
        const bool active = unc <= cl || (ratio >= 1.f - clip && ratio <= 1.f + clip);
        const float glp = active ? -adv * ratio / (float)B : 0.f;   // d loss / d log pi
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float var = __expf(2.f * s[i]);
            const float d = a[i] - mn[i];
            d_mu[3 * (size_t)row + i] = glp * d / var;
            ds[i] = glp * (d * d / var - 1.f);
            const float dm = mo[i] - mn[i];
            kl += s[i] - so[i] + (__expf(2.f * so[i]) + dm * dm) / (2.f * var) - 0.5f;
        }
        const float dv = v_new[row] - ret;
        d_v[row] = 2.f * vf_coef * dv / (float)B;
        vl = dv * dv;
    }
    float vals[6] = {ds[0], ds[1], ds[2], pol, vl, kl};
    block_sums<6>(vals, lpart + 8 * (size_t)blockIdx.x);   // summed in order by loss_sums
}

// the loss block sums in order: log-std gradient into d_std[0..2], policy loss,
// value loss and KL into their minibatch sums
__global__ void loss_sums_kernel(const float* __restrict__ lpart, int P, float* __restrict__ d_std,
                                 float* __restrict__ scal) {
    if (threadIdx.x != 0) return;
    float t[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int j = 0; j < P; ++j)
#pragma unroll
        for (int k = 0; k < 6; ++k) t[k] += lpart[8 * (size_t)j + k];
    d_std[0] += t[0]; d_std[1] += t[1]; d_std[2] += t[2];
    scal[S_POL] += t[3]; scal[S_VAL] += t[4]; scal[S_KL] += t[5];
}

// minibatch scalars: mean KL -> learning rate (App. L rule), entropy term of the log-std gradient,
// global norm -> clip scale; accumulations for the statistics; per-minibatch sums cleared
__global__ void finalize_kernel(int B, float ent_coef, float kl_target, float max_norm, float* __restrict__ d_std,
                                float* __restrict__ scal) {
    if (threadIdx.x != 0) return;
    const float kl = scal[S_KL] / (float)B;
    float lr = scal[S_LR];
    if (kl > 2.f * kl_target) lr = fmaxf(kLrMin, lr * 0.5f);
    else if (kl < 0.5f * kl_target) lr = fminf(kLrMax, lr * 2.f);
    scal[S_LR] = lr;
    float sq = scal[S_SUMSQ];
    for (int i = 0; i < 3; ++i) {
        d_std[i] -= ent_coef;   // d(-c_e H)/d s_i = -c_e
        sq += d_std[i] * d_std[i];
    }
    const float norm = sqrtf(sq);
    scal[S_SCALE] = norm > max_norm ? max_norm / (norm + 1e-6f) : 1.f;
    scal[S_ACC_POL] += scal[S_POL] / (float)B;
    scal[S_ACC_VAL] += scal[S_VAL] / (float)B;
    scal[S_ACC_KL] += kl;
    scal[S_ACC_NORM] += norm;
    scal[S_POL] = scal[S_VAL] = scal[S_KL] = scal[S_SUMSQ] = 0.f;
}

// Adam on the 3 log standard deviations; clears their gradient
__global__ void adam_std_kernel(float* __restrict__ s, float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, const float* __restrict__ scal, float c1, float c2) {
    const int i = threadIdx.x;
    if (i >= 3) return;
    const float gi = g[i] * scal[S_SCALE];
    const float mi = 0.9f * m[i] + 0.1f * gi, vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    s[i] -= scal[S_LR] * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    g[i] = 0.f;
}

unsigned grid_for(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct sf_ppo {
    sf_handle h = nullptr;
    sf_mlp_handle actor = nullptr, critic = nullptr;
    // the late-fusion mode: the paper's network on the full observation (W = 1929, group counts)
    sf_lf_handle lf = nullptr;
    LfTrainer* lft = nullptr;
    int W = kObsW;
    int32_t *nr = nullptr, *nv = nullptr, *g_nr = nullptr, *g_nv = nullptr;
    float *obs_boot = nullptr, *mu_boot = nullptr;      // the bootstrap state's observation, a scratch mean
    int32_t *nr_boot = nullptr, *nv_boot = nullptr;
    sf_ppo_config cfg{};
    cudaStream_t st = nullptr;
    // MLP mode: the critic's rollout forward runs beside the actor's on a second stream
    // (forked from and joined back to st by events)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    std::string err;
    int A = 0, T = 0, B = 0;               // agents, horizon, minibatch rows
    unsigned long long steps = 0;          // control steps sampled so far (the sampling counter)
    unsigned long long updates = 0;
    int std_t = 0;                         // Adam step of the log-stds
    std::vector<void*> allocs;
    float *obs = nullptr, *act = nullptr, *mu = nullptr, *logp = nullptr, *val = nullptr, *rew = nullptr;
    uint8_t* done = nullptr;
    float *adv = nullptr, *ret = nullptr;
    float *log_std = nullptr, *log_std_old = nullptr, *g_std = nullptr, *m_std = nullptr, *v_std = nullptr;
    float* scal = nullptr;
    double* moments = nullptr;
    float* lpart = nullptr;     // [blocks of a minibatch][8] loss block sums
    double* mpart = nullptr;    // [blocks of the agents][2] advantage moment block sums
    float* rpart = nullptr;     // [kSumBlocks] rollout reward block sums
    float *g_obs = nullptr, *g_small = nullptr, *mu_new = nullptr, *v_new = nullptr, *d_mu = nullptr, *d_v = nullptr;
    bool collected = false;
};

// the world handle's stream and library-owned outputs (sf_api.cu)
cudaStream_t sf_handle_stream(sf_handle h);

namespace {

sf_status pfail(sf_ppo* p, sf_status s, const std::string& e) {
    if (p) p->err = e;
    return s;
}

// the two networks of either mode: rollout inference of A rows (val may be null
// with the MLPs; mu is required), the training forward, backward, gradient norm
// and Adam of the minibatch
sf_status nets_infer(sf_ppo* p, const float* obs, const int32_t* nr, const int32_t* nv, float* mu, float* val) {
    if (p->lft) return sf_lf_forward_on(p->lf, p->st, obs, nr, nv, p->A, mu, val, nullptr);
    const bool both = mu && val && p->aux;
    if (both && (cudaEventRecord(p->ev[0], p->st) != cudaSuccess || cudaStreamWaitEvent(p->aux, p->ev[0], 0) != cudaSuccess))
        return SF_ERR_CUDA;
    sf_status s = mu ? sf_mlp_forward_on(p->actor, p->st, obs, kObsW, p->A, mu, 3) : SF_OK;
    if (s == SF_OK && val) s = sf_mlp_forward_on(p->critic, both ? p->aux : p->st, obs, kObsW, p->A, val, 1);
    if (both && (cudaEventRecord(p->ev[1], p->aux) != cudaSuccess || cudaStreamWaitEvent(p->st, p->ev[1], 0) != cudaSuccess))
        return SF_ERR_CUDA;
    return s;
}
sf_status nets_train_forward(sf_ppo* p, int B) {
    if (p->lft) return lft_forward(p->lft, p->g_obs, p->g_nr, p->g_nv, B, p->mu_new, p->v_new);
    // the critic reads the actor's bf16 copy of the minibatch (converted once); the two
    // forwards then run side by side (the critic's on aux)
    sf_status s = sf_mlp_convert_train_on(p->actor, p->st, p->g_obs, kObsW, B);
    const bool fork = s == SF_OK && p->aux != nullptr;
    if (fork && (cudaEventRecord(p->ev[0], p->st) != cudaSuccess || cudaStreamWaitEvent(p->aux, p->ev[0], 0) != cudaSuccess))
        return SF_ERR_CUDA;
    if (s == SF_OK) s = sf_mlp_forward_converted_on(p->actor, p->st, B, p->mu_new, 3);
    if (s == SF_OK) s = sf_mlp_forward_train_shared_on(p->critic, p->actor, fork ? p->aux : p->st, B, p->v_new, 1);
    if (fork && (cudaEventRecord(p->ev[1], p->aux) != cudaSuccess || cudaStreamWaitEvent(p->st, p->ev[1], 0) != cudaSuccess))
        return SF_ERR_CUDA;
    return s;
}
sf_status nets_backward(sf_ppo* p, int B) {
    sf_status s;
    if (p->lft) {
        s = lft_backward(p->lft, p->d_mu, p->d_v, B);
        if (s == SF_OK) s = lft_grad_sumsq(p->lft, p->scal + S_SUMSQ);
        return s;
    }
    // the two backward passes are independent: the critic's runs beside the actor's on aux;
    // the gradient norm (one accumulator) follows the join
    const bool fork = p->aux != nullptr;
    if (fork && (cudaEventRecord(p->ev[0], p->st) != cudaSuccess || cudaStreamWaitEvent(p->aux, p->ev[0], 0) != cudaSuccess))
        return SF_ERR_CUDA;
    s = sf_mlp_backward_on(p->actor, p->st, p->d_mu, 3, B);
    if (s == SF_OK) s = sf_mlp_backward_on(p->critic, fork ? p->aux : p->st, p->d_v, 1, B);
    if (fork && (cudaEventRecord(p->ev[1], p->aux) != cudaSuccess || cudaStreamWaitEvent(p->st, p->ev[1], 0) != cudaSuccess))
        return SF_ERR_CUDA;
    if (s == SF_OK) s = sf_mlp_grad_sumsq_on(p->actor, p->st, p->scal + S_SUMSQ);
    if (s == SF_OK) s = sf_mlp_grad_sumsq_on(p->critic, p->st, p->scal + S_SUMSQ);
    return s;
}
sf_status nets_adam(sf_ppo* p) {
    if (p->lft) return lft_adam(p->lft, p->scal + S_LR, p->scal + S_SCALE);
    sf_status s = sf_mlp_adam_on(p->actor, p->st, p->scal + S_LR, p->scal + S_SCALE);
    if (s == SF_OK) s = sf_mlp_adam_on(p->critic, p->st, p->scal + S_LR, p->scal + S_SCALE);
    return s;
}

template <class T>
bool palloc(sf_ppo* p, T** ptr, size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T) + 64) != cudaSuccess) return false;
    p->allocs.push_back(q);
    cudaMemset(q, 0, count * sizeof(T) + 64);
    *ptr = static_cast<T*>(q);
    return true;
}

unsigned long long gcd_ull(unsigned long long a, unsigned long long b) {
    while (b) { const unsigned long long t = a % b; a = b; b = t; }
    return a;
}

}  // namespace

extern "C" {

void sf_ppo_default_config(sf_ppo_config* c) {
    if (!c) return;
    *c = sf_ppo_config{};
    c->horizon = 128;
    c->minibatches = 16;
    c->epochs = 5;
    c->lr = 2.09e-4f;
    c->kl_target = 0.01f;
    c->gamma = 0.99f;
    c->lam = 0.98f;
    c->clip = 0.15f;
    c->ent_coef = 3e-5f;
    c->vf_coef = 1.0f;
    c->max_grad_norm = 1.0f;
    c->init_log_std = 0.0f;
    c->dt = 1.0f / 30.0f;
    c->substeps = 4;
    c->seed = 0x5CE7EFAC;
}

const char* sf_ppo_last_error(sf_ppo_handle p) { return p ? p->err.c_str() : "NULL handle"; }

sf_status sf_ppo_create(sf_handle h, sf_mlp_handle actor, sf_mlp_handle critic, const sf_ppo_config* cfg,
                        sf_ppo_handle* out) {
    if (!h || !actor || !critic || !cfg || !out) return SF_ERR_INVALID_ARG;
    *out = nullptr;
    const int A = sf_num_agents(h);
    if (A <= 0) return SF_ERR_STATE;
    if (sf_mlp_in_dim(actor) != kObsW || sf_mlp_out_dim(actor) != 3 || sf_mlp_in_dim(critic) != kObsW ||
        sf_mlp_out_dim(critic) != 1)
        return SF_ERR_INVALID_ARG;
    const sf_ppo_config& c = *cfg;
    if (c.horizon < 1 || c.minibatches < 1 || c.epochs < 1 || !(c.lr > 0.f) || !(c.kl_target > 0.f) ||
        c.substeps < 1 || !(c.dt > 0.f))
        return SF_ERR_INVALID_ARG;
    const size_t N = (size_t)A * c.horizon;
    const int B = (int)((N / c.minibatches) / 8 * 8);   // minibatch rows (a multiple of 8; the remainder is unused)
    if (B < 8) return SF_ERR_INVALID_ARG;
    sf_ppo* p = new sf_ppo();
    p->h = h; p->actor = actor; p->critic = critic; p->cfg = c;
    p->st = sf_handle_stream(h);
    p->A = A; p->T = c.horizon; p->B = B;
    const size_t T = (size_t)c.horizon;
    bool ok = palloc(p, &p->obs, T * A * kObsW) && palloc(p, &p->act, T * A * 3) && palloc(p, &p->mu, T * A * 3) &&
              palloc(p, &p->logp, T * A) && palloc(p, &p->val, (T + 1) * A) && palloc(p, &p->rew, T * A) &&
              palloc(p, &p->done, T * A) && palloc(p, &p->adv, T * A) && palloc(p, &p->ret, T * A) &&
              palloc(p, &p->log_std, 3) && palloc(p, &p->log_std_old, 3) && palloc(p, &p->g_std, 3) &&
              palloc(p, &p->m_std, 3) && palloc(p, &p->v_std, 3) && palloc(p, &p->scal, S_COUNT) &&
              palloc(p, &p->moments, 2) && palloc(p, &p->g_obs, (size_t)B * kObsW) &&
              palloc(p, &p->lpart, (size_t)grid_for(B) * 8) && palloc(p, &p->mpart, (size_t)grid_for(A) * 2) &&
              palloc(p, &p->rpart, (size_t)kSumBlocks) &&
              palloc(p, &p->g_small, (size_t)B * 12) && palloc(p, &p->mu_new, (size_t)B * 3) &&
              palloc(p, &p->v_new, (size_t)B) && palloc(p, &p->d_mu, (size_t)B * 3) && palloc(p, &p->d_v, (size_t)B);
    if (ok) ok = sf_mlp_reserve(actor, std::max(A, B)) == SF_OK && sf_mlp_reserve(critic, std::max(A, B)) == SF_OK;
    if (ok) ok = cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; i < 2 && ok; ++i) ok = cudaEventCreateWithFlags(&p->ev[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        for (void* q : p->allocs) cudaFree(q);
        for (cudaEvent_t ev : p->ev)
            if (ev) cudaEventDestroy(ev);
        if (p->aux) cudaStreamDestroy(p->aux);
        delete p;
        return SF_ERR_OOM;
    }
    const float s0[3] = {c.init_log_std, c.init_log_std, c.init_log_std};
    float sc[S_COUNT] = {0};
    sc[S_LR] = c.lr;
    sc[S_SCALE] = 1.f;
    cudaMemcpy(p->log_std, s0, 12, cudaMemcpyHostToDevice);
    cudaMemcpy(p->scal, sc, sizeof(sc), cudaMemcpyHostToDevice);
    *out = p;
    return SF_OK;
}

sf_status sf_ppo_create_lf(sf_handle h, sf_lf_handle lf, const sf_ppo_config* cfg, sf_ppo_handle* out) {
    if (!h || !lf || !cfg || !out) return SF_ERR_INVALID_ARG;
    *out = nullptr;
    const int A = sf_num_agents(h);
    if (A <= 0) return SF_ERR_STATE;
    const sf_ppo_config& c = *cfg;
    if (c.horizon < 1 || c.minibatches < 1 || c.epochs < 1 || !(c.lr > 0.f) || !(c.kl_target > 0.f) ||
        c.substeps < 1 || !(c.dt > 0.f))
        return SF_ERR_INVALID_ARG;
    const size_t N = (size_t)A * c.horizon;
    const int B = (int)((N / c.minibatches) / 8 * 8);
    if (B < 8) return SF_ERR_INVALID_ARG;
    sf_ppo* p = new sf_ppo();
    p->h = h; p->lf = lf; p->cfg = c;
    p->st = sf_handle_stream(h);
    p->A = A; p->T = c.horizon; p->B = B;
    p->W = SF_FULL_OBS_DIM;
    const size_t T = (size_t)c.horizon, W = (size_t)p->W;
    bool ok = palloc(p, &p->obs, T * A * W) && palloc(p, &p->nr, T * A) && palloc(p, &p->nv, T * A) &&
              palloc(p, &p->act, T * A * 3) && palloc(p, &p->mu, T * A * 3) && palloc(p, &p->logp, T * A) &&
              palloc(p, &p->val, (T + 1) * A) && palloc(p, &p->rew, T * A) && palloc(p, &p->done, T * A) &&
              palloc(p, &p->adv, T * A) && palloc(p, &p->ret, T * A) && palloc(p, &p->log_std, 3) &&
              palloc(p, &p->log_std_old, 3) && palloc(p, &p->g_std, 3) && palloc(p, &p->m_std, 3) &&
              palloc(p, &p->v_std, 3) && palloc(p, &p->scal, S_COUNT) && palloc(p, &p->moments, 2) &&
              palloc(p, &p->g_obs, (size_t)B * W) && palloc(p, &p->g_nr, (size_t)B) && palloc(p, &p->g_nv, (size_t)B) &&
              palloc(p, &p->obs_boot, (size_t)A * W) && palloc(p, &p->nr_boot, (size_t)A) &&
              palloc(p, &p->nv_boot, (size_t)A) && palloc(p, &p->mu_boot, (size_t)A * 3) &&
              palloc(p, &p->lpart, (size_t)grid_for(B) * 8) && palloc(p, &p->mpart, (size_t)grid_for(A) * 2) &&
              palloc(p, &p->rpart, (size_t)kSumBlocks) && palloc(p, &p->g_small, (size_t)B * 12) &&
              palloc(p, &p->mu_new, (size_t)B * 3) && palloc(p, &p->v_new, (size_t)B) &&
              palloc(p, &p->d_mu, (size_t)B * 3) && palloc(p, &p->d_v, (size_t)B);
    if (ok) ok = sf_lf_reserve(lf, A) == SF_OK && lft_create(lf, p->st, &p->lft) == SF_OK;
    if (!ok) {
        lft_destroy(p->lft);
        for (void* q : p->allocs) cudaFree(q);
        delete p;
        return SF_ERR_OOM;
    }
    // the policy's log standard deviations start from the network's own (its last 3 parameters)
    std::vector<float> prm(sf_lf_num_params());
    float s0[3] = {c.init_log_std, c.init_log_std, c.init_log_std};
    if (sf_lf_get_params(lf, prm.data(), prm.size()) == SF_OK)
        for (int i = 0; i < 3; ++i) s0[i] = prm[prm.size() - 3 + i];
    float sc[S_COUNT] = {0};
    sc[S_LR] = c.lr;
    sc[S_SCALE] = 1.f;
    cudaMemcpy(p->log_std, s0, 12, cudaMemcpyHostToDevice);
    cudaMemcpy(p->scal, sc, sizeof(sc), cudaMemcpyHostToDevice);
    *out = p;
    return SF_OK;
}

sf_status sf_ppo_lf_grads(sf_ppo_handle p, const float* d_obs, const int32_t* d_n_road, const int32_t* d_n_veh,
                          int rows, const float* d_dmean, const float* d_dvalue, float* d_mean, float* d_value,
                          uint16_t* d_argmax, float* h_grads, size_t n) {
    if (!p || !p->lft || !d_obs || !d_n_road || !d_n_veh || !d_dmean || !d_dvalue || !h_grads ||
        n != sf_lf_num_params() || rows < 8 || rows % 8)
        return SF_ERR_INVALID_ARG;
    float* mu = d_mean;
    float* v = d_value;
    if (!mu || !v) {   // the rollout-sized scratch would not hold more than A rows: use the minibatch buffers
        if (rows > p->B) return pfail(p, SF_ERR_INVALID_ARG, "sf_ppo_lf_grads: rows above the minibatch size need outputs");
        if (!mu) mu = p->mu_new;
        if (!v) v = p->v_new;
    }
    sf_status s = lft_forward(p->lft, d_obs, d_n_road, d_n_veh, rows, mu, v);
    if (s == SF_OK) s = lft_backward(p->lft, d_dmean, d_dvalue, rows);
    if (s == SF_OK && d_argmax) s = lft_argmax(p->lft, d_argmax);
    if (s == SF_OK) s = lft_get(p->lft, nullptr, h_grads);
    if (s != SF_OK) return pfail(p, s, std::string("sf_ppo_lf_grads: ") + lft_error(p->lft));
    h_grads[n - 3] = h_grads[n - 2] = h_grads[n - 1] = 0.f;
    return SF_OK;
}

sf_status sf_ppo_lf_params(sf_ppo_handle p, float* h_params, size_t n) {
    if (!p || !p->lft || !h_params || n != sf_lf_num_params()) return SF_ERR_INVALID_ARG;
    sf_status s = lft_get(p->lft, h_params, nullptr);
    if (s != SF_OK) return pfail(p, s, std::string("sf_ppo_lf_params: ") + lft_error(p->lft));
    return cudaMemcpy(h_params + n - 3, p->log_std, 12, cudaMemcpyDeviceToHost) == cudaSuccess ? SF_OK : SF_ERR_CUDA;
}

sf_status sf_ppo_destroy(sf_ppo_handle p) {
    if (!p) return SF_OK;
    cudaStreamSynchronize(p->st);
    if (p->aux) cudaStreamSynchronize(p->aux);
    for (cudaEvent_t ev : p->ev)
        if (ev) cudaEventDestroy(ev);
    if (p->aux) cudaStreamDestroy(p->aux);
    lft_destroy(p->lft);
    for (void* q : p->allocs) cudaFree(q);
    delete p;
    return SF_OK;
}

sf_status sf_ppo_collect(sf_ppo_handle p) {
    if (!p) return SF_ERR_INVALID_ARG;
    sf_outputs o{};
    sf_status s = sf_output_ptrs(p->h, &o);
    if (s != SF_OK) return pfail(p, s, "sf_ppo_collect: world outputs");
    const int A = p->A;
    cudaError_t e = cudaMemcpyAsync(p->log_std_old, p->log_std, 12, cudaMemcpyDeviceToDevice, p->st);
    for (int t = 0; t < p->T && e == cudaSuccess; ++t) {
        float* obs_t = p->obs + (size_t)t * A * p->W;
        int32_t *nr_t = nullptr, *nv_t = nullptr;
        if (p->lft) {   // the full observation (App. D) of the current state and its group counts
            nr_t = p->nr + (size_t)t * A;
            nv_t = p->nv + (size_t)t * A;
            s = sf_observe_full(p->h, obs_t, nr_t, nv_t, nullptr, nullptr);
            if (s != SF_OK) return pfail(p, s, std::string("sf_ppo_collect: observation: ") + sf_last_error(p->h));
        } else {
            e = cudaMemcpyAsync(obs_t, o.obs, (size_t)A * kObsW * 4, cudaMemcpyDeviceToDevice, p->st);
            if (e != cudaSuccess) break;
        }
        s = nets_infer(p, obs_t, nr_t, nv_t, p->mu + (size_t)t * A * 3, p->val + (size_t)t * A);
        if (s != SF_OK) return pfail(p, s, "sf_ppo_collect: policy / value forward");
        sample_kernel<<<grid_for(A), 256, 0, p->st>>>(p->mu + (size_t)t * A * 3, p->log_std, A, p->cfg.seed,
                                                       p->steps, p->act + (size_t)t * A * 3, p->logp + (size_t)t * A);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        ++p->steps;
        s = sf_step(p->h, p->act + (size_t)t * A * 3, p->cfg.dt, p->cfg.substeps);
        if (s != SF_OK) return pfail(p, s, std::string("sf_ppo_collect: step: ") + sf_last_error(p->h));
        record_step_kernel<<<grid_for(A), 256, 0, p->st>>>(o.reward, o.done, A, p->rew + (size_t)t * A,
                                                           p->done + (size_t)t * A);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {   // the value of the state after the last step bootstraps GAE
        if (p->lft) {
            s = sf_observe_full(p->h, p->obs_boot, p->nr_boot, p->nv_boot, nullptr, nullptr);
            if (s == SF_OK)
                s = nets_infer(p, p->obs_boot, p->nr_boot, p->nv_boot, p->mu_boot, p->val + (size_t)p->T * A);
        } else {
            s = nets_infer(p, o.obs, nullptr, nullptr, nullptr, p->val + (size_t)p->T * A);
        }
        if (s != SF_OK) return pfail(p, s, "sf_ppo_collect: bootstrap value");
    }
    if (e != cudaSuccess) return pfail(p, SF_ERR_CUDA, std::string("sf_ppo_collect: ") + cudaGetErrorString(e));
    p->collected = true;
    return SF_OK;
}

sf_status sf_ppo_update(sf_ppo_handle p, float* h_stats) {
    if (!p) return SF_ERR_INVALID_ARG;
    struct EndShare {   // on every exit: the critic stops reading the actor's input copy
        sf_mlp_handle m;
        ~EndShare() { sf_mlp_end_share(m); }
    } end_share{p->critic};
    if (!p->collected) return pfail(p, SF_ERR_STATE, "sf_ppo_update: no rollout collected");
    const int A = p->A, T = p->T, B = p->B;
    const size_t N = (size_t)A * T;
    const sf_ppo_config& c = p->cfg;
    cudaError_t e = cudaMemsetAsync(p->scal + S_ACC_POL, 0, 4 * 4, p->st);
    if (e == cudaSuccess) {
        gae_kernel<<<grid_for(A), 256, 0, p->st>>>(p->rew, p->done, p->val, T, A, c.gamma, c.lam, p->adv, p->ret,
                                                    p->mpart);
        parts_final_kernel<double><<<1, 32, 0, p->st>>>(p->mpart, (int)grid_for(A), 2, 2, p->moments, false);
        normalise_kernel<<<grid_for(N), 256, 0, p->st>>>(p->adv, N, p->moments);
        sum_part_kernel<<<kSumBlocks, 256, 0, p->st>>>(p->rew, N, p->rpart);   // the rollout's reward sum
        parts_final_kernel<float><<<1, 32, 0, p->st>>>(p->rpart, kSumBlocks, 1, 1, p->scal + S_REW, false);
        e = cudaGetLastError();
    }
    int nmb = 0;
    for (int ep = 0; ep < c.epochs && e == cudaSuccess; ++ep) {
        // a fresh affine bijection of the rows for this epoch: (mul i + add) mod N with gcd(mul, N) = 1
        unsigned long long h0 = (unsigned long long)c.seed * 0x9E3779B97F4A7C15ull + (p->updates * 131 + ep) * 7919;
        auto mix = [](unsigned long long x) {
            x += 0x9E3779B97F4A7C15ull;
            x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
            x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
            return x ^ (x >> 31);
        };
        Perm pm{};
        pm.n = N;
        pm.mul = mix(h0) % N;
        while (pm.mul == 0 || gcd_ull(pm.mul, N) != 1) pm.mul = (pm.mul + 1) % N;
        pm.add = mix(h0 + 1) % N;
        for (int mb = 0; mb < c.minibatches && e == cudaSuccess; ++mb) {
            gather_kernel<<<grid_for((size_t)B * 32), 256, 0, p->st>>>(pm, (size_t)mb * B, B, p->W, p->obs, p->act,
                                                                        p->mu, p->logp, p->adv, p->ret, p->g_obs,
                                                                        p->g_small, p->nr, p->nv, p->g_nr, p->g_nv);
            e = cudaGetLastError();
            if (e != cudaSuccess) break;
            sf_status s = nets_train_forward(p, B);
            if (s != SF_OK) return pfail(p, s, "sf_ppo_update: forward");
            loss_grad_kernel<<<grid_for(B), 256, 0, p->st>>>(B, p->g_small, p->mu_new, p->v_new, p->log_std,
                                                              p->log_std_old, c.clip, c.vf_coef, p->d_mu, p->d_v,
                                                              p->lpart);
            loss_sums_kernel<<<1, 32, 0, p->st>>>(p->lpart, (int)grid_for(B), p->g_std, p->scal);
            e = cudaGetLastError();
            if (e != cudaSuccess) break;
            s = nets_backward(p, B);
            if (s != SF_OK) return pfail(p, s, "sf_ppo_update: backward");
            finalize_kernel<<<1, 32, 0, p->st>>>(B, c.ent_coef, c.kl_target, c.max_grad_norm, p->g_std, p->scal);
            s = nets_adam(p);
            if (s != SF_OK) return pfail(p, s, "sf_ppo_update: Adam");
            ++p->std_t;
            const float c1 = 1.f - std::pow(0.9f, (float)p->std_t), c2 = 1.f - std::pow(0.999f, (float)p->std_t);
            adam_std_kernel<<<1, 32, 0, p->st>>>(p->log_std, p->g_std, p->m_std, p->v_std, p->scal, c1, c2);
            e = cudaGetLastError();
            ++nmb;
        }
    }
    ++p->updates;
    if (e == cudaSuccess && p->lft) {   // the rollout's network takes the trained dense layers
        const sf_status s = lft_publish(p->lft);
        if (s != SF_OK) return pfail(p, s, std::string("sf_ppo_update: ") + lft_error(p->lft));
    }
    if (e != cudaSuccess) return pfail(p, SF_ERR_CUDA, std::string("sf_ppo_update: ") + cudaGetErrorString(e));
    if (h_stats) {
        float sc[S_COUNT];
        e = cudaMemcpyAsync(sc, p->scal, sizeof(sc), cudaMemcpyDeviceToHost, p->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
        if (e != cudaSuccess) return pfail(p, SF_ERR_CUDA, std::string("sf_ppo_update: ") + cudaGetErrorString(e));
        h_stats[0] = sc[S_REW] / (float)N;
        h_stats[1] = sc[S_ACC_POL] / (float)nmb;
        h_stats[2] = sc[S_ACC_VAL] / (float)nmb;
        h_stats[3] = sc[S_ACC_KL] / (float)nmb;
        h_stats[4] = sc[S_LR];
        h_stats[5] = sc[S_ACC_NORM] / (float)nmb;
    }
    return SF_OK;
}

sf_status sf_ppo_log_std(sf_ppo_handle p, float* h_log_std) {
    if (!p || !h_log_std) return SF_ERR_INVALID_ARG;
    cudaStreamSynchronize(p->st);
    return cudaMemcpy(h_log_std, p->log_std, 12, cudaMemcpyDeviceToHost) == cudaSuccess ? SF_OK : SF_ERR_CUDA;
}

sf_status sf_ppo_rollout_ptrs(sf_ppo_handle p, sf_ppo_rollout* r) {
    if (!p || !r) return SF_ERR_INVALID_ARG;
    r->obs = p->obs; r->actions = p->act; r->mean = p->mu; r->logp = p->logp; r->value = p->val;
    r->reward = p->rew; r->done = p->done; r->advantage = p->adv; r->ret = p->ret;
    r->horizon = p->T; r->num_agents = p->A; r->minibatch_rows = p->B;
    return SF_OK;
}

sf_status sf_ppo_loss_grads(sf_ppo_handle p, const float* d_obs, const float* d_small, int rows, float* d_mean,
                            float* d_value, float* d_dmean, float* d_dvalue, float* h_out) {
    if (!p || !d_obs || !d_small || rows < 8 || rows % 8 || rows > p->B || !h_out) return SF_ERR_INVALID_ARG;
    if (p->lft) return pfail(p, SF_ERR_STATE, "sf_ppo_loss_grads: an MLP-mode call (this engine trains the late-fusion network)");
    const sf_ppo_config& c = p->cfg;
    float* mu = d_mean ? d_mean : p->mu_new;
    float* v = d_value ? d_value : p->v_new;
    sf_status s = sf_mlp_forward_train_on(p->actor, p->st, d_obs, kObsW, rows, mu, 3);
    if (s == SF_OK) s = sf_mlp_forward_train_on(p->critic, p->st, d_obs, kObsW, rows, v, 1);
    if (s != SF_OK) return pfail(p, s, "sf_ppo_loss_grads: forward");
    cudaError_t e = cudaMemsetAsync(p->g_std, 0, 12, p->st);
    float keep[S_COUNT];
    if (e == cudaSuccess) e = cudaMemcpyAsync(keep, p->scal, sizeof(keep), cudaMemcpyDeviceToHost, p->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
    if (e == cudaSuccess) {
        loss_grad_kernel<<<grid_for(rows), 256, 0, p->st>>>(rows, d_small, mu, v, p->log_std, p->log_std_old, c.clip,
                                                             c.vf_coef, d_dmean ? d_dmean : p->d_mu,
                                                             d_dvalue ? d_dvalue : p->d_v, p->lpart);
        loss_sums_kernel<<<1, 32, 0, p->st>>>(p->lpart, (int)grid_for(rows), p->g_std, p->scal);
        e = cudaGetLastError();
    }
    float sc[S_COUNT], gs[3];
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc, p->scal, sizeof(sc), cudaMemcpyDeviceToHost, p->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gs, p->g_std, 12, cudaMemcpyDeviceToHost, p->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
    if (e == cudaSuccess) e = cudaMemcpy(p->scal, keep, sizeof(keep), cudaMemcpyHostToDevice);   // no side effects
    if (e == cudaSuccess) e = cudaMemset(p->g_std, 0, 12);
    if (e != cudaSuccess) return pfail(p, SF_ERR_CUDA, std::string("sf_ppo_loss_grads: ") + cudaGetErrorString(e));
    h_out[0] = gs[0] - c.ent_coef; h_out[1] = gs[1] - c.ent_coef; h_out[2] = gs[2] - c.ent_coef;
    h_out[3] = (sc[S_POL] - keep[S_POL]) / (float)rows;
    h_out[4] = (sc[S_VAL] - keep[S_VAL]) / (float)rows;
    h_out[5] = (sc[S_KL] - keep[S_KL]) / (float)rows;
    return SF_OK;
}

}  // extern "C"
