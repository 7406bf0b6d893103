// sf_lf.cu -- the paper's late-fusion actor-critic network (SceneFactory App. E)
// on the sm_103a tensor cores.
//
// Each of the two networks (actor, critic; no shared weights) encodes the
// 1,929-value observation (App. D) by groups:
//   ego      11 -> 64 -> 64 (ELU)                          tc GEMMs (sf_gemm.cu)
//   road     5 -> 96 -> 96 (ELU) per slot, masked max-pool  lf_set_kernel below
//   vehicles 7 -> 96 -> 96 (ELU) per slot, masked max-pool  lf_set_kernel below
//   trunk    [ego | road | vehicles] 256 -> 128 -> 64 (ELU), then the actor's
//            3 action means or the critic's value (linear)    tc GEMMs
// The max-pool is masked by the group's count (the observation fills a prefix
// of the slots); an empty group pools to zeros.
//
// lf_set_kernel runs the encoder of one group over work items of 32
// consecutive agents: two persistent CTAs of 8 warps per SM, even CTAs the
// actor's network, odd ones the critic's (each holds its network's weights in
// shared memory and 256 TMEM columns).  An item's slots are concatenated into
// tiles of 128 rows, each agent's filled slots padded to a multiple of 8 rows
// (an 8-row group belongs to one agent):
//   gather   rows -> bf16 A1 [128 slots][16 inputs] (swizzled smem; the
//            layer-1 bias rides on input 15 = 1), the next tile's global loads
//            issued before this tile's epilogues
//   MMA 1    D1[128 slots][96] = A1 . W1^T              (K = 16)
//   epi 1    ELU -> bf16 H1[128 slots][96]              (K-major for MMA 2)
//   MMA 2    D2[128 features][128 slots] = W2 . H1^T    (K = 96; features
//            96..127 are zero rows of the weight image)
//   epi 2    each thread owns one feature and walks the tile's slot columns:
//            a running max, flushed to the item's pool (shared atomicMax on
//            order-preserving integer keys) at every agent boundary
// after the item: pooled max + bias -> ELU -> bf16 into the trunk inputs.
// ELU is monotone and the bias is constant per feature, so max-then-activate
// equals the paper's activate-then-max.  Every mbarrier wait is bounded (1 s).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sf.h"
#include "sf_gemm.cuh"
#include "sf_mlp_internal.cuh"
#include "sf_tc.cuh"

namespace {

using namespace sftc;

constexpr int kEgo = 11, kKR = 350, kPT = 5, kKV = 24, kNB = 7;
constexpr int kObs = kEgo + kKR * kPT + kKV * kNB;   // 1929
constexpr int kRoad0 = kEgo, kVeh0 = kEgo + kKR * kPT;
constexpr int kHid = 96;                             // set-encoder width
constexpr int kG = 32;                               // agents per work item
constexpr int kThreads = 256;
constexpr unsigned kLfTimeout = 4u;                  // error-word bit: a bounded wait gave up

// shared memory of one CTA (one network), offsets from a 1024-byte aligned base
constexpr int kOffW1 = 0;                           // [96 rows][128 B]: layer 1, K 0..15 used (bias at K 15)
constexpr int kOffW2 = kOffW1 + 96 * 128;           // 12288: 2 K-atoms of [128 rows][128 B], rows 96..127 zero
constexpr int kImgBytes = kOffW2 + 2 * 128 * 128;   // 45056: one network's weight image
constexpr int kOffA1 = kImgBytes;                   // [128 slots][128 B]
constexpr int kOffH1 = kOffA1 + 128 * 128;          // 61440: 2 K-atoms of [128 slots][128 B]
constexpr int kOffPool = kOffH1 + 2 * 128 * 128;    // 94208: u32 [kG][96]
constexpr int kMaxGroups = kG * ((kKR + 7) / 8);    // 1408 8-row groups of an item at most
constexpr int kOffMeta = kOffPool + kG * kHid * 4;  // 106496: u32 [kMaxGroups] group words
constexpr int kOffMisc = kOffMeta + kMaxGroups * 4; // 112128
constexpr int kMiscBytes = 1024;
constexpr int kSmemBytes = kOffMisc + kMiscBytes + 1024;   // 114176: two CTAs per SM
// the training variant pools 64-bit keys (value, then the lowest slot) for items of
// kGTrain agents, in the 32-bit pool's space: two CTAs per SM as in inference
constexpr int kGTrain = 16;
static_assert(kGTrain * kHid * 8 <= kG * kHid * 4, "the training pool must fit the inference pool's space");
constexpr uint32_t kTmemCols = 256;                 // D1 at column 0 (96), D2 at column 128 (128)

struct SetArgs {
    const float* obs;          // [A][ld]
    int ld, off, F, K;         // row stride, group offset, features per slot, slots
    const int32_t* count;      // [A] filled slots
    int num_agents;
    const uint4* wimg;         // 2 x kImgBytes: actor then critic weight images (bf16, swizzled)
    const float* b2;           // [2][96] layer-2 biases (layer-1 biases are in the images)
    __nv_bfloat16* xa;         // [A][ldx] actor trunk input (may be null in the training variant)
    __nv_bfloat16* xc;         // [A][ldx] critic trunk input
    int ldx, xoff;             // columns [xoff, xoff + 96) receive the pooled embedding
    unsigned* err;
    // training variant only: per network n (actor 0, critic 1), the fp32 pooled
    // embedding xf + n * xf_net [A][ldxf] (columns xoff..), the pooled
    // pre-activation maximum pmax + n * A * 96 and its slot amax (0xFFFF: empty group)
    float* xf;
    size_t xf_net;
    int ldxf;
    float* pmax;
    uint16_t* amax;
};

__device__ __forceinline__ uint32_t fkey(float f) {   // order-preserving float -> u32 (0 is below every key)
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float funkey(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}
__device__ __forceinline__ float elu(float x) { return x > 0.f ? x : __expf(x) - 1.f; }
// maximum of three values in one instruction (NaN inputs are ignored as by fmaxf)
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// the agent (item-local) whose rows contain item row r: last s with rs[s] <= r
__device__ __forceinline__ int agent_of_row(const int* rs, int r) {
    int lo = 0, hi = kG - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rs[mid] <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// the word of an item's 8-row group: filled rows (1..8) in bits 0-7, the agent
// (item-local; kG past the item) in bits 8-15, the agent's slot of the group's
// first row in bits 16-31; written once per item, read by the gathers and the
// max-pool of every tile
__device__ __forceinline__ uint32_t group_word(int s, int slot0, int valid) {
    return (uint32_t)valid | ((uint32_t)s << 8) | ((uint32_t)slot0 << 16);
}
constexpr uint32_t kPastItem = (uint32_t)kG << 8;

// features of item row (tile * 128 + row) into v[0..7] (zeros past F, past the agent's filled
// slots or past the item); returns whether the row is a filled slot
__device__ __forceinline__ bool gather_row(const SetArgs& a, const uint32_t* meta, int a0, int total, int tile,
                                           int row, float (&v)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = 0.f;
    const int r = tile * 128 + row;
    if (r >= total) return false;
    const uint32_t md = meta[r >> 3];
    const int k = r & 7;
    if (k >= (int)(md & 0xFFu)) return false;
    const int al = (int)((md >> 8) & 0xFFu), slot = (int)(md >> 16) + k;
    const float* src = a.obs + (size_t)(a0 + al) * a.ld + a.off + (size_t)slot * a.F;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (i < a.F) v[i] = __ldg(src + i);
    return true;
}

// Two CTAs per SM; even CTAs run the actor's encoder, odd ones the critic's.
// The training variant also keeps, for every pooled feature, the slot that
// holds the maximum (the lowest one on ties), on items of kGTrain agents.
template <bool TRAIN>
__global__ void __launch_bounds__(kThreads, 2) lf_set_kernel(const SetArgs a) {
    constexpr int G = TRAIN ? kGTrain : kG;   // agents per item
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(sm);
    uint32_t* pool = reinterpret_cast<uint32_t*>(sm + kOffPool);
    unsigned long long* pool64 = reinterpret_cast<unsigned long long*>(sm + kOffPool);   // TRAIN only
    uint32_t* meta = reinterpret_cast<uint32_t*>(sm + kOffMeta);
    int* rs = reinterpret_cast<int*>(sm + kOffMisc);                       // [kG + 1] item row starts (x8)
    int* cnt = reinterpret_cast<int*>(sm + kOffMisc + 640);               // [kG] filled slots per agent
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffMisc + 192);     // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kOffMisc + 208);
    float* sb2 = reinterpret_cast<float*>(sm + kOffMisc + 256);           // [96]
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kOffMisc + 212);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int net = blockIdx.x & 1, cta = blockIdx.x >> 1, ncta = gridDim.x >> 1;

    // ---- weights, bias, pool, barriers, TMEM
    const uint4* img = a.wimg + (size_t)net * (kImgBytes / 16);
    for (int i = tid; i < kImgBytes / 16; i += kThreads) reinterpret_cast<uint4*>(sm)[i] = __ldg(img + i);
    for (int i = tid; i < kHid; i += kThreads) sb2[i] = __ldg(a.b2 + net * kHid + i);
    for (int i = tid; i < G * kHid; i += kThreads) {
        if (TRAIN) pool64[i] = 0ull;
        else pool[i] = 0u;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t kIdesc1 = instr_desc(128, kHid), kIdesc2 = instr_desc(128, 128);
    uint32_t phase1 = 0, phase2 = 0;
    bool ok = true;   // false once any thread's bounded wait gave up (checked once per tile)
    const int q = warp & 3, hh = warp >> 2;                 // TMEM lane quarter, column half of this warp
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    __nv_bfloat16* X = net ? a.xc : a.xa;
    const int num_items = (a.num_agents + G - 1) / G;

    for (int item = cta; item < num_items && ok; item += ncta) {
        const int a0 = item * G;
        const int na = min(G, a.num_agents - a0);
        if (warp == 0) {   // each agent's slots take a multiple of 8 rows: an 8-row group is one agent's
            const int n = lane < na ? min(max(__ldg(a.count + a0 + lane), 0), a.K) : 0;
            int n8 = (n + 7) & ~7;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xFFFFFFFFu, n8, o);
                if (lane >= o) n8 += t;
            }
            rs[lane + 1] = n8;
            cnt[lane] = n;
            if (lane == 0) rs[0] = 0;
        }
        __syncthreads();
        const int total = rs[kG];
        const int ntiles = (total + 127) / 128;
        for (int g = tid; g < total / 8; g += kThreads) {
            const int s = agent_of_row(rs, 8 * g), slot0 = 8 * g - rs[s];
            meta[g] = group_word(s, slot0, min(8, cnt[s] - slot0));
        }
        __syncthreads();
        float v8[8];
        bool live = gather_row(a, meta, a0, total, 0, tid >> 1, v8);
        for (int t = 0; t < ntiles; ++t) {
            // ---- A1: 128 slots x 16 inputs (features, zeros, 1 at K 15 for the bias), two threads per row
            {
                const int row = tid >> 1, half = tid & 1;
                const uint4 w = half == 0 ? make_uint4(pack_bf16(v8[0], v8[1]), pack_bf16(v8[2], v8[3]),
                                                       pack_bf16(v8[4], v8[5]), pack_bf16(v8[6], v8[7]))
                                          : make_uint4(0u, 0u, 0u, live ? 0x3F800000u : 0u);
                *reinterpret_cast<uint4*>(sm + kOffA1 + swz128(row, half)) = w;
            }
            fence_async_smem();
            ok = __syncthreads_and(*abort_flag == 0) != 0;   // also: the last tile's TMEM reads are done
            if (!ok) break;
            tc_after();
            if (tid == 0) {
                umma_bf16(tmem, smem_desc(sbase + kOffA1), smem_desc(sbase + kOffW1), kIdesc1, 0u);
                umma_commit(&bar[0]);
            }
            if (t + 1 < ntiles) live = gather_row(a, meta, a0, total, t + 1, tid >> 1, v8);   // in flight meanwhile

            // ---- epilogue 1: ELU -> bf16 rows of H1 (this warp: its 32 slots, 48 of the 96 columns)
            // every lane waits, then the warp reconverges (the tcgen05.ld that follows is warp-synchronous)
            if (!__all_sync(0xFFFFFFFFu, mbar_wait(&bar[0], phase1, a.err, kLfTimeout))) *abort_flag = 1;
            phase1 ^= 1u;
            tc_after();
            {
                uint32_t r0[32], r1[16];
                tmem_ld32_async(tmem + lanes + (uint32_t)(48 * hh), r0);
                tmem_ld16_async(tmem + lanes + (uint32_t)(48 * hh + 32), r1);
                tmem_wait();
                tmem_hold(r0);
                tmem_hold(r1);
                const int row = 32 * q + lane;
                unsigned char* h1 = sm + kOffH1;
#pragma unroll
                for (int u = 0; u < 6; ++u) {    // 8 columns -> one 16-byte chunk of the K-major row
                    uint32_t p[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int c = 8 * u + 2 * e;
                        p[e] = c < 32 ? elu_bf16x2(r0[c], r0[c + 1]) : elu_bf16x2(r1[c - 32], r1[c - 31]);
                    }
                    const int j = 6 * hh + u;    // chunk of the 96-wide row
                    *reinterpret_cast<uint4*>(h1 + (j >> 3) * 16384 + swz128(row, j & 7)) = make_uint4(p[0], p[1], p[2], p[3]);
                }
            }
            fence_async_smem();
            tc_before();
            __syncthreads();
            if (tid == 0) {
                tc_after();
#pragma unroll
                for (int kk = 0; kk < 6; ++kk) {
                    const uint64_t ad = smem_desc(sbase + kOffW2 + (kk >> 2) * 16384) + 2 * (kk & 3);
                    const uint64_t bd = smem_desc(sbase + kOffH1 + (kk >> 2) * 16384) + 2 * (kk & 3);
                    umma_bf16(tmem + 128, ad, bd, kIdesc2, kk > 0 ? 1u : 0u);
                }
                umma_commit(&bar[1]);
            }

            // ---- epilogue 2: per feature, running max over 64 of the tile's slot columns
            if (!__all_sync(0xFFFFFFFFu, mbar_wait(&bar[1], phase2, a.err, kLfTimeout))) *abort_flag = 1;
            phase2 ^= 1u;
            tc_after();
            const int rbase = 128 * t + 64 * hh;
            if (q < 3 && rbase < total) {
                uint32_t r[2][32];
                tmem_ld32_async(tmem + lanes + (uint32_t)(128 + 64 * hh), r[0]);
                tmem_ld32_async(tmem + lanes + (uint32_t)(128 + 64 * hh + 32), r[1]);
                // the words of these columns' eight 8-row groups, read while the TMEM loads run
                const int g0 = rbase >> 3, ng = total >> 3;
                uint32_t md[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) md[i] = g0 + i < ng ? meta[g0 + i] : kPastItem;
                tmem_wait();
                tmem_hold(r[0]);
                tmem_hold(r[1]);
                const int f = 32 * q + lane;
                int cur = -1;                            // agent of the running max
                float m = -INFINITY;
                int msl = 0;                             // TRAIN: the slot of the running max
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int s = (int)((md[i] >> 8) & 0xFFu), valid = (int)(md[i] & 0xFFu);
                    if (s != cur) {                      // warp-uniform: the group starts the next agent
                        if (cur >= 0 && cur < kG) {
                            if (TRAIN)
                                atomicMax(&pool64[cur * kHid + f],
                                          ((unsigned long long)fkey(m) << 32) | (unsigned long long)(0xFFFF - msl));
                            else
                                atomicMax(&pool[cur * kHid + f], fkey(m));
                        }
                        cur = s;
                        m = -INFINITY;
                    }
                    if (s >= kG) continue;               // rows past the item
                    const uint32_t* v = r[i >> 2] + 8 * (i & 3);
                    float x[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) x[k] = __uint_as_float(v[k]);
                    if (TRAIN) {                         // slots in increasing order: strict > keeps the first maximum
                        const int slot0 = (int)(md[i] >> 16);
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            if (k < valid && x[k] > m) { m = x[k]; msl = slot0 + k; }
                    } else {
                        if (valid < 8) {                 // warp-uniform: the agent's last, partly filled group
#pragma unroll
                            for (int k = 1; k < 8; ++k) x[k] = k < valid ? x[k] : x[0];
                        }
                        m = max3f(max3f(m, x[0], x[1]), max3f(x[2], x[3], x[4]), max3f(x[5], x[6], x[7]));
                    }
                }
                if (cur >= 0 && cur < kG) {              // continues past these rows
                    if (TRAIN)
                        atomicMax(&pool64[cur * kHid + f],
                                  ((unsigned long long)fkey(m) << 32) | (unsigned long long)(0xFFFF - msl));
                    else
                        atomicMax(&pool[cur * kHid + f], fkey(m));
                }
            }
            tc_before();   // this tile's TMEM reads before the next tile's barrier and MMAs
        }
        if (!ok) break;
        __syncthreads();
        if (*abort_flag) break;
        // ---- the item's pooled embeddings: + bias, ELU, bf16 into the trunk inputs
        for (int i = tid; i < na * kHid; i += kThreads) {
            const int al = i / kHid, col = i - al * kHid;
            if (TRAIN) {
                const unsigned long long k = pool64[i];
                pool64[i] = 0ull;
                const float pm = k ? funkey((uint32_t)(k >> 32)) : 0.f;
                const float y = k ? elu(pm + sb2[col]) : 0.f;
                const size_t row = (size_t)(a0 + al);
                if (X) X[row * a.ldx + a.xoff + col] = __float2bfloat16_rn(y);
                a.xf[net * a.xf_net + row * a.ldxf + a.xoff + col] = y;
                a.pmax[((size_t)net * a.num_agents + row) * kHid + col] = pm;
                a.amax[((size_t)net * a.num_agents + row) * kHid + col] =
                    k ? (uint16_t)(0xFFFF - (uint32_t)(k & 0xFFFFull)) : (uint16_t)0xFFFF;
            } else {
                const uint32_t k = pool[i];
                pool[i] = 0u;
                const float y = k ? elu(funkey(k) + sb2[col]) : 0.f;
                X[(size_t)(a0 + al) * a.ldx + a.xoff + col] = __float2bfloat16_rn(y);
            }
        }
        __syncthreads();
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// ego features -> bf16 [A][16] (11 used)
__global__ void lf_ego_kernel(const float* __restrict__ obs, int ld, int A, __nv_bfloat16* __restrict__ x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A * 16) return;
    const int a = i >> 4, j = i & 15;
    x[i] = __float2bfloat16_rn(j < kEgo ? obs[(size_t)a * ld + j] : 0.f);
}

// bf16 trunk inputs of both nets -> fp32 [A][512]
__global__ void lf_embed_kernel(const __nv_bfloat16* __restrict__ xa, const __nv_bfloat16* __restrict__ xc, int A,
                                float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A * 512) return;
    const int a = i >> 9, j = i & 511;
    out[i] = __bfloat162float(j < 256 ? xa[(size_t)a * 256 + j] : xc[(size_t)a * 256 + j - 256]);
}

// ------------------------------------------------------------------ set-encoder backward (training)
// Gradient of one group's encoder (W1 [96][F], b1, W2 [96][96], b2) for each
// network from the gradient of its pooled embedding.  The pooled feature f of
// a sample is y_f = ELU(z2max_f + b2_f), z2max_f the layer-2 pre-activation of
// the slot s_f holding the maximum (recorded by the training forward), so
//   dp_f = dy_f ELU'(z2max_f + b2_f),  db2_f += dp_f,  dW2[f][.] += dp_f h1(s_f),
//   dh1(s)[.] = sum over f with s_f = s of dp_f W2[f][.],
//   dz1(s) = dh1(s) ELU'(z1(s)),  dW1 += dz1(s) x(s)^T,  db1 += dz1(s).
// Only the distinct maximising slots of a sample carry a gradient, and they
// become the rows of dense products on the tensor cores: row (b, j) is sample
// b's j-th distinct maximising slot (ascending), X its bf16 inputs with 1 at
// column 15, dZ2 its row of dp_f over the features f whose maximum it holds
// (zeros elsewhere).  Over the R rows of a minibatch:
//   z1 = X W1b^T, H1 = ELU(z1)   W1b: bf16 W1 with the bf16 b1 at column 15 (the forward's
//                                 image); K = 16, so on the CUDA cores, fp32 sums
//   dH1 = dZ2 W2,  dZ1 = dH1 * ELU'(z1)
//   [dW2 | db2] = dZ2^T [H1 | 1],   [dW1 | . | db1] = dZ1^T X
// The two weight-gradient products reduce over the rows with split K, their
// partials added in split order, so the result repeats bit for bit.
constexpr int kSlotWords = (kKR + 31) / 32;   // bitmap words of a sample's slots
constexpr int kLdW2 = 104;                    // row stride of the [dW2 | db2] partials (97 used)
constexpr int kBackSplit = 148;               // split-K partials of the weight gradients at most

struct BackRows {
    const float* obs;          // [B][ld] the minibatch's observations
    int ld, off, F, K;         // row stride, group offset, features per slot, slots
    const int32_t* count;      // [B]
    int B;
    const float* theta;        // per network: the group's masters [W1 (96 x F) | b1 | W2 (96 x 96) | b2]
    size_t theta_net;          // distance between the two networks' masters
    const float* pmax;         // [2][B][96] pooled pre-activation maxima
    const uint16_t* amax;      // [2][B][96] their slots (0xFFFF: empty group)
    const float* dx;           // [2][B][lddx] gradient of the trunk input (columns xoff..)
    size_t dx_net;
    int lddx, xoff;
    int* nd;                   // [2][B] distinct maximising slots of each sample
    int* offs;                 // [2][B + 1] their first row (exclusive prefix sum); [B]: R
};

// the bitmap of sample b's valid maximising slots (network net) in words[0..kSlotWords), one warp
__device__ __forceinline__ void slot_bitmap(const BackRows& a, int net, int b, int n, int lane, unsigned* words) {
    if (lane < kSlotWords) words[lane] = 0u;
    __syncwarp();
    const uint16_t* am = a.amax + ((size_t)net * a.B + b) * kHid;
    for (int f = lane; f < kHid; f += 32) {
        const int s = am[f];
        if (s < n) atomicOr(&words[s >> 5], 1u << (s & 31));
    }
    __syncwarp();
}

// distinct maximising slots per (sample, network): one warp per sample, networks on grid y
__global__ void __launch_bounds__(256) lfb_count_kernel(const BackRows a) {
    __shared__ unsigned words[8][kSlotWords + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, net = blockIdx.y;
    const int b = blockIdx.x * 8 + warp;
    if (b >= a.B) return;   // warp-uniform
    const int n = min(max(a.count[b], 0), a.K);
    slot_bitmap(a, net, b, n, lane, words[warp]);
    const int d = __reduce_add_sync(0xFFFFFFFFu, lane < kSlotWords ? __popc(words[warp][lane]) : 0);
    if (lane == 0) a.nd[(size_t)net * a.B + b] = d;
}

// first row of every sample (exclusive prefix sum of the counts, samples in order)
// and the total R, per network (one block each, 1024 samples a pass, loads coalesced)
__global__ void __launch_bounds__(1024) lfb_scan_kernel(const int* __restrict__ nd, int B, int* __restrict__ offs) {
    __shared__ int wsum[32];
    __shared__ int tile_total;
    const int net = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int* d = nd + (size_t)net * B;
    int* o = offs + (size_t)net * (B + 1);
    int carry = 0;
    for (int base = 0; base < B; base += 1024) {
        const int i = base + t;
        const int v = i < B ? d[i] : 0;
        int incl = v;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const int u = __shfl_up_sync(0xFFFFFFFFu, incl, k);
            if (lane >= k) incl += u;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            const int x = wsum[lane];
            int ix = x;
#pragma unroll
            for (int k = 1; k < 32; k <<= 1) {
                const int u = __shfl_up_sync(0xFFFFFFFFu, ix, k);
                if (lane >= k) ix += u;
            }
            wsum[lane] = ix - x;
            if (lane == 31) tile_total = ix;
        }
        __syncthreads();
        if (i < B) o[i] = carry + wsum[w] + incl - v;
        carry += tile_total;
        __syncthreads();   // wsum and tile_total are rewritten by the next pass
    }
    if (t == 0) o[B] = carry;
}

// the row buffers of one network's products (ldR: row stride of the transposed ones)
struct BackBufs {
    __nv_bfloat16* x;      // [R][16]   inputs, 1 at column 15
    __nv_bfloat16* xt;     // [16][ldR]
    __nv_bfloat16* dz2;    // [R][96]
    __nv_bfloat16* dz2t;   // [96][ldR]
    __nv_bfloat16* h1t;    // [97][ldR] H1^T (the tensor cores write rows 0..95), row 96: ones
    __nv_bfloat16* dh1t;   // [96][ldR]
    __nv_bfloat16* dz1t;   // [96][ldR]
    __nv_bfloat16* w1b;    // [96][16]
    __nv_bfloat16* w2t;    // [96 hidden][96 features]: W2 transposed
    int ldR;
};

// the rows of network net's products: one warp per sample writes its slots' inputs (X,
// X^T) and the ones row of H1^T; the block's 8 samples own a contiguous range of rows,
// whose dZ2 and dZ2^T (dp_f in the row of f's slot, zeros elsewhere) are staged in
// shared memory kRowChunk rows at a time and written out with consecutive threads on
// consecutive elements
constexpr int kRowChunk = 192;
constexpr int kTileLd = kRowChunk + 2;   // bf16 stride of the staged dZ2^T rows (97 words: no bank conflicts)
__global__ void __launch_bounds__(256) lfb_rows_kernel(const BackRows a, const BackBufs o, int net) {
    __shared__ unsigned words[8][kSlotWords + 1];
    __shared__ int wpre[8][kSlotWords + 1];   // set bits before each word
    __shared__ int rank[8][kHid];             // feature -> row of its slot within the sample (-1: none)
    __shared__ float dpv[8][kHid];            // feature -> dp
    __shared__ int slot[8][kHid];             // row within the sample -> slot
    __shared__ int s_r0[8], s_d[8];
    __shared__ __nv_bfloat16 tile[kHid][kTileLd];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int b = blockIdx.x * 8 + warp;
    const int n = b < a.B ? min(max(a.count[b], 0), a.K) : 0;
    const int ldR = o.ldR;
    int D = 0;
    if (n > 0) {   // warp-uniform
        slot_bitmap(a, net, b, n, lane, words[warp]);
        if (lane == 0) {
            int c = 0;
            for (int w = 0; w < kSlotWords; ++w) {
                wpre[warp][w] = c;
                c += __popc(words[warp][w]);
            }
            wpre[warp][kSlotWords] = c;
        }
        __syncwarp();
        D = wpre[warp][kSlotWords];
        const size_t bi = ((size_t)net * a.B + b) * kHid;
        const float* b2 = a.theta + (size_t)net * a.theta_net + kHid * a.F + kHid + kHid * kHid;
        const float* dy = a.dx + (size_t)net * a.dx_net + (size_t)b * a.lddx + a.xoff;
        for (int f = lane; f < kHid; f += 32) {
            const int s = a.amax[bi + f];
            int r = -1;
            float d = 0.f;
            if (s < n) {
                const float u = a.pmax[bi + f] + b2[f];
                d = dy[f] * (u > 0.f ? 1.f : expf(u));
                r = wpre[warp][s >> 5] + __popc(words[warp][s >> 5] & ((1u << (s & 31)) - 1u));
                slot[warp][r] = s;   // every feature of the slot writes the same value
            }
            rank[warp][f] = r;
            dpv[warp][f] = d;
        }
        __syncwarp();
        const int r0 = a.offs[(size_t)net * (a.B + 1) + b];
        if (lane == 0) s_r0[warp] = r0;
        for (int j = lane; j < D; j += 32) {   // lanes: rows
            const size_t row = (size_t)r0 + j;
            const float* src = a.obs + (size_t)b * a.ld + a.off + (size_t)slot[warp][j] * a.F;
            float x[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) x[k] = 0.f;
#pragma unroll
            for (int k = 0; k < 7; ++k)
                if (k < a.F) x[k] = src[k];
            x[15] = 1.f;
            uint4* xr = reinterpret_cast<uint4*>(o.x + row * 16);
            xr[0] = make_uint4(pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]), pack_bf16(x[4], x[5]), pack_bf16(x[6], x[7]));
            xr[1] = make_uint4(pack_bf16(x[8], x[9]), pack_bf16(x[10], x[11]), pack_bf16(x[12], x[13]),
                               pack_bf16(x[14], x[15]));
#pragma unroll
            for (int k = 0; k < 16; ++k) o.xt[(size_t)k * ldR + row] = __float2bfloat16_rn(x[k]);
            o.h1t[(size_t)kHid * ldR + row] = __float2bfloat16_rn(1.f);
        }
    }
    if (lane == 0) s_d[warp] = D;
    // the block's rows [rb0, rb1): its samples' first rows in order
    const int bb0 = min(blockIdx.x * 8, a.B), bb1 = min(blockIdx.x * 8 + 8, a.B);
    const int rb0 = a.offs[(size_t)net * (a.B + 1) + bb0], rb1 = a.offs[(size_t)net * (a.B + 1) + bb1];
    __syncthreads();
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    for (int c0 = rb0; c0 < rb1; c0 += kRowChunk) {
        const int cw = min(kRowChunk, rb1 - c0);
        for (int f = warp; f < kHid; f += 8)
            for (int c = lane; c < cw; c += 32) tile[f][c] = zero;
        __syncthreads();
        for (int w = 0; w < 8; ++w) {                 // every (sample, feature): dp into its row
            if (s_d[w] == 0) continue;                 // block-uniform
            const int f = tid;
            if (f >= kHid) continue;
            const int r = rank[w][f];
            if (r < 0) continue;
            const int c = s_r0[w] + r - c0;
            if (c >= 0 && c < cw) tile[f][c] = __float2bfloat16_rn(dpv[w][f]);
        }
        __syncthreads();
        for (int f = warp; f < kHid; f += 8)           // dZ2^T: lanes on consecutive columns
            for (int c = lane; c < cw; c += 32) o.dz2t[(size_t)f * ldR + c0 + c] = tile[f][c];
        for (int c = warp; c < cw; c += 8)             // dZ2: lanes on consecutive features of a row
            for (int f = lane; f < kHid; f += 32) o.dz2[((size_t)c0 + c) * kHid + f] = tile[f][c];
        __syncthreads();
    }
}

// zeros in the padding columns [R, ldR) of X^T (16 rows), dZ2^T (96) and the ones row of
// H1^T (its other rows are written with dZ1^T), one block per row
__global__ void lfb_pad_kernel(BackBufs o, int R) {
    const int row = blockIdx.x, c = R + threadIdx.x;
    if (c >= o.ldR) return;
    __nv_bfloat16* p = row < 16 ? o.xt + (size_t)row * o.ldR
                     : row < 16 + kHid ? o.dz2t + (size_t)(row - 16) * o.ldR
                                       : o.h1t + (size_t)kHid * o.ldR;
    p[c] = __float2bfloat16_rn(0.f);
}

// the bf16 operands of one network's weights: W1b [96][16] (W1, zeros, the layer-1 bias
// at column 15, the forward's image) and W2 transposed
__global__ void lfb_weights_kernel(const float* __restrict__ th, int F, __nv_bfloat16* __restrict__ w1b,
                                   __nv_bfloat16* __restrict__ w2t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kHid * 16) {
        const int h = i >> 4, k = i & 15;
        const float v = k < F ? th[h * F + k] : (k == 15 ? th[kHid * F + h] : 0.f);
        w1b[i] = __float2bfloat16_rn(v);
    } else if (i < kHid * 16 + kHid * kHid) {
        const int e = i - kHid * 16, h = e / kHid, f = e - h * kHid;
        w2t[e] = __float2bfloat16_rn(th[kHid * F + kHid + f * kHid + h]);
    }
}

// H1^T = bf16(ELU(z1)) and dZ1^T = bf16(dH1 * ELU'(z1)) with z1 = X W1b^T recomputed in
// fp32 from the bf16 inputs and weights (K = 16: a CUDA-core job), two rows a thread
// (4-byte accesses; lanes hold consecutive rows, so every store is contiguous across the
// warp); columns [R, ldR) get zeros
__global__ void __launch_bounds__(256) lfb_h1dz1_kernel(BackBufs o, int R) {
    __shared__ float w[kHid][16];
    for (int i = threadIdx.x; i < kHid * 16; i += blockDim.x) w[i >> 4][i & 15] = __bfloat162float(o.w1b[i]);
    __syncthreads();
    const int r = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (r >= o.ldR) return;
    const size_t ld = (size_t)o.ldR;
    float x[2][16];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
#pragma unroll
        for (int k = 0; k < 16; ++k) x[q][k] = 0.f;
        if (r + q < R) {
            const uint4* xr = reinterpret_cast<const uint4*>(o.x + (size_t)(r + q) * 16);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const uint4 u = xr[c];
                const uint32_t p[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    x[q][8 * c + 2 * e] = __uint_as_float(p[e] << 16);
                    x[q][8 * c + 2 * e + 1] = __uint_as_float(p[e] & 0xFFFF0000u);
                }
            }
        }
    }
#pragma unroll 2
    for (int h = 0; h < kHid; ++h) {
        const uint32_t gp = *reinterpret_cast<const uint32_t*>(o.dh1t + h * ld + r);
        float hv[2], dv[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            float z = 0.f;
#pragma unroll
            for (int k = 0; k < 16; ++k) z = fmaf(x[q][k], w[h][k], z);
            const float e = z > 0.f ? 1.f : expf(z);
            const float g = __uint_as_float(q ? (gp & 0xFFFF0000u) : (gp << 16));
            const bool in = r + q < R;
            hv[q] = in ? (z > 0.f ? z : e - 1.f) : 0.f;
            dv[q] = in ? g * e : 0.f;
        }
        *reinterpret_cast<uint32_t*>(o.h1t + h * ld + r) = pack_bf16(hv[0], hv[1]);
        *reinterpret_cast<uint32_t*>(o.dz1t + h * ld + r) = pack_bf16(dv[0], dv[1]);
    }
}

// the weight-gradient partials added in split order, into the masters' layout
// [W1 (96 x F) | b1 | W2 (96 x 96) | b2]: ws1 [S1][96][16] ([dW1 | . | db1]),
// ws2 [S2][96][kLdW2] ([dW2 | db2])
__global__ void lfb_reduce_kernel(const float* __restrict__ ws1, int S1, const float* __restrict__ ws2, int S2, int F,
                                  float* __restrict__ g) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int nW1 = kHid * F, nW2 = kHid * kHid;
    if (e >= nW1 + kHid + nW2 + kHid) return;
    const float* p;
    int S;
    size_t stride;
    if (e < nW1 + kHid) {
        const int h = e < nW1 ? e / F : e - nW1, k = e < nW1 ? e - h * F : 15;
        p = ws1 + h * 16 + k; S = S1; stride = (size_t)kHid * 16;
    } else {
        const int q = e - nW1 - kHid;
        const int f = q < nW2 ? q / kHid : q - nW2, h = q < nW2 ? q - f * kHid : kHid;
        p = ws2 + f * kLdW2 + h; S = S2; stride = (size_t)kHid * kLdW2;
    }
    float acc = 0.f;
    for (int s = 0; s < S; ++s) acc += p[s * stride];
    g[e] = acc;
}

// The inference images of both networks' set encoders from the masters:
// layer 1 as bf16 [96 rows][K 16] with the bias at K 15, layer 2 as [128 rows][K 96]
// (K-major 128-byte swizzled atoms of 64 columns), and the layer-2 biases
__global__ void lf_image_kernel(const float* __restrict__ theta, size_t theta_net, int F, unsigned char* __restrict__ img,
                                float* __restrict__ sb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   // (net, row, column) of the two layers
    const int per = kHid * 16 + kHid * kHid + kHid;
    if (i >= 2 * per) return;
    const int net = i / per, e = i - net * per;
    const float* th = theta + (size_t)net * theta_net;
    unsigned char* base = img + (size_t)net * kImgBytes;
    auto put = [&](int off, int rows_total, int r, int k, float v) {
        const int atom = k / 64, kk = k % 64;
        const size_t o = (size_t)off + (size_t)atom * rows_total * 128 + (size_t)r * 128 +
                         (size_t)((((kk / 8) ^ (r & 7)) * 16) + (kk % 8) * 2);
        *reinterpret_cast<__nv_bfloat16*>(base + o) = __float2bfloat16_rn(v);
    };
    if (e < kHid * 16) {                                   // layer 1: inputs 0..F-1, zeros, the bias at K 15
        const int r = e / 16, k = e % 16;
        const float v = k < F ? th[r * F + k] : (k == 15 ? th[kHid * F + r] : 0.f);
        put(kOffW1, 96, r, k, v);
    } else if (e < kHid * 16 + kHid * kHid) {
        const int t = e - kHid * 16, r = t / kHid, k = t % kHid;
        put(kOffW2, 128, r, k, th[kHid * F + kHid + t]);
    } else {
        const int j = e - kHid * 16 - kHid * kHid;
        sb[net * kHid + j] = th[kHid * F + kHid + kHid * kHid + j];
    }
}

// Adam (0.9, 0.999, 1e-8) over the set encoders' masters, gradients scaled by *scale
__global__ void lf_adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                               float* __restrict__ v, size_t n, const float* __restrict__ lr,
                               const float* __restrict__ scale, float c1, float c2) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i] * *scale;
    const float mi = 0.9f * m[i] + 0.1f * gi, vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= *lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// sum of squares of g[0, n): per-block partials (fixed order), then one thread adds them in order to *acc
constexpr int kSqBlocks = 128;
__global__ void lf_sumsq_part_kernel(const float* __restrict__ g, size_t n, float* __restrict__ part) {
    __shared__ float red[256];
    float s = 0.f;
    for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (size_t)gridDim.x * 256) s += g[i] * g[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void lf_sumsq_final_kernel(const float* __restrict__ part, int k, float* __restrict__ acc) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < k; ++i) s += part[i];
        *acc += s;
    }
}

// ------------------------------------------------------------------ host side
struct Layer {   // one dense layer of a net in the oracle's parameter order
    int out, in;
};
const Layer kLayers[9] = {{64, 11}, {64, 64}, {96, 5}, {96, 96}, {96, 7}, {96, 96}, {128, 256}, {64, 128}, {0, 64}};
enum { L_EGO0, L_EGO1, L_ROAD0, L_ROAD1, L_VEH0, L_VEH1, L_TRUNK0, L_TRUNK1, L_HEAD };

size_t net_params(int head) {
    size_t n = 0;
    for (int l = 0; l < 9; ++l) {
        const int o = l == L_HEAD ? head : kLayers[l].out;
        n += (size_t)o * kLayers[l].in + o;
    }
    return n;
}
size_t total_params() { return net_params(3) + net_params(1) + 3; }

uint16_t to_bf16(float f) {   // round to nearest even
    uint32_t b;
    std::memcpy(&b, &f, 4);
    if ((b & 0x7F800000u) == 0x7F800000u) return (uint16_t)(b >> 16);
    b += 0x7FFFu + ((b >> 16) & 1u);
    return (uint16_t)(b >> 16);
}

}  // namespace

struct sf_lf {
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<float> params;           // oracle layout, fp32
    std::vector<void*> allocs;           // parameters and the error word
    std::vector<void*> acts;             // activation buffers (grown on demand)
    // device parameters
    uint4* img[2] = {nullptr, nullptr};  // road, vehicles: 2 x kImgBytes each (actor, critic)
    float* sb[2] = {nullptr, nullptr};   // road, vehicles: layer-2 biases [2][96]
    __nv_bfloat16* w[2][6] = {};         // per net: ego0 [64][16], ego1, trunk0, trunk1, head [out][64] (bf16)
    float* b[2][6] = {};                 // their biases
    // activations (grown on demand)
    int cap = 0;
    __nv_bfloat16 *xego = nullptr, *he1[2] = {nullptr, nullptr}, *x[2] = {nullptr, nullptr};
    __nv_bfloat16 *t1 = nullptr, *t1c = nullptr;   // trunk layer 1 outputs (actor, critic)
    unsigned* d_err = nullptr;
    // the critic's ego and trunk GEMM chains run beside the actor's on a second stream
    // (forked from and joined back to the caller's stream by events; parallel branches
    // when captured into a graph)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

sf_status lfail(sf_lf* m, sf_status s, const std::string& msg) {
    if (m) m->err = msg;
    return s;
}

template <class T>
bool lalloc(sf_lf* m, T** p, size_t count, bool act = false) {
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess) return false;
    (act ? m->acts : m->allocs).push_back(q);
    *p = static_cast<T*>(q);
    return true;
}

// swizzled bf16 image of a [rows][k_used] weight block as K-major 128-byte atoms of 64 columns
void put_swizzled(std::vector<uint16_t>& img, size_t base, int rows_total, int r, int k, float v) {
    const int atom = k / 64, kk = k % 64;
    const size_t off = base + (size_t)atom * rows_total * 128 + (size_t)r * 128 +
                       (size_t)((((kk / 8) ^ (r & 7)) * 16) + (kk % 8) * 2);
    img[off / 2] = to_bf16(v);
}

sf_status upload(sf_lf* m) {
    const float* P = m->params.data();
    size_t k = 0;
    std::vector<const float*> W[2], B[2];
    for (int n = 0; n < 2; ++n)
        for (int l = 0; l < 9; ++l) {
            const int o = l == L_HEAD ? (n == 0 ? 3 : 1) : kLayers[l].out, i = kLayers[l].in;
            W[n].push_back(P + k); k += (size_t)o * i;
            B[n].push_back(P + k); k += o;
        }
    cudaError_t e = cudaSuccess;
    // set-encoder images: group g (0 road, 1 vehicles) uses layers (ROAD0, ROAD1) / (VEH0, VEH1); per
    // network, layer 1 as [96 rows][K 16] with the bias at K 15 and layer 2 as [128 rows][K 96]
    for (int g = 0; g < 2; ++g) {
        const int l0 = g == 0 ? L_ROAD0 : L_VEH0, l1 = l0 + 1, F = kLayers[l0].in;
        std::vector<uint16_t> img(kImgBytes, 0);   // two networks of kImgBytes bytes
        std::vector<float> bb(2 * kHid);
        for (int n = 0; n < 2; ++n) {
            const size_t base = (size_t)n * kImgBytes;
            for (int j = 0; j < kHid; ++j) {
                for (int f = 0; f < F; ++f) put_swizzled(img, base + kOffW1, 96, j, f, W[n][l0][j * F + f]);
                put_swizzled(img, base + kOffW1, 96, j, 15, B[n][l0][j]);
                for (int f = 0; f < kHid; ++f) put_swizzled(img, base + kOffW2, 128, j, f, W[n][l1][j * kHid + f]);
                bb[n * kHid + j] = B[n][l1][j];
            }
        }
        if (e == cudaSuccess) e = cudaMemcpy(m->img[g], img.data(), 2 * kImgBytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(m->sb[g], bb.data(), 2 * kHid * 4, cudaMemcpyHostToDevice);
    }
    // dense layers (bf16 [out][in_padded]) of the tc GEMMs
    const int dl[5] = {L_EGO0, L_EGO1, L_TRUNK0, L_TRUNK1, L_HEAD};
    for (int n = 0; n < 2; ++n)
        for (int t = 0; t < 5; ++t) {
            const int l = dl[t], o = l == L_HEAD ? (n == 0 ? 3 : 1) : kLayers[l].out, i = kLayers[l].in;
            const int ip = l == L_EGO0 ? 16 : (i + 7) / 8 * 8;   // ego input padded to 16
            std::vector<uint16_t> wb((size_t)o * ip, 0);
            for (int r = 0; r < o; ++r)
                for (int c = 0; c < i; ++c) wb[(size_t)r * ip + c] = to_bf16(W[n][l][(size_t)r * i + c]);
            if (e == cudaSuccess) e = cudaMemcpy(m->w[n][t], wb.data(), wb.size() * 2, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(m->b[n][t], B[n][l], (size_t)o * 4, cudaMemcpyHostToDevice);
        }
    if (e != cudaSuccess) return lfail(m, SF_ERR_CUDA, std::string("sf_lf_set_params: ") + cudaGetErrorString(e));
    return SF_OK;
}

sf_status ensure(sf_lf* m, int A) {
    if (A <= m->cap) return SF_OK;
    cudaDeviceSynchronize();   // the buffers may be in use on any stream the network ran on
    for (void* p : m->acts) cudaFree(p);
    m->acts.clear();
    m->cap = 0;
    const size_t Aa = (size_t)A;
    bool okk = lalloc(m, &m->xego, Aa * 16, true) && lalloc(m, &m->he1[0], Aa * 64, true) &&
               lalloc(m, &m->he1[1], Aa * 64, true) && lalloc(m, &m->x[0], Aa * 256, true) &&
               lalloc(m, &m->x[1], Aa * 256, true) && lalloc(m, &m->t1, Aa * 128, true) &&
               lalloc(m, &m->t1c, Aa * 128, true);
    if (!okk) return lfail(m, SF_ERR_OOM, "sf_lf_forward: cudaMalloc of the activations failed");
    m->cap = A;
    return SF_OK;
}

cudaError_t gemm(sf_lf* m, cudaStream_t st, const __nv_bfloat16* A, const __nv_bfloat16* B, const float* bias, int M,
                 int N, int K, int act, float* out_f32, __nv_bfloat16* out_bf16, int ldc) {
    GemmArgs g{};
    g.A = A; g.B = B; g.bias = bias;
    g.out_f32 = out_f32; g.out_bf16 = out_bf16;
    g.M = M; g.N = N; g.Nb = N; g.K = K;
    g.ldc = ldc; g.ldt = 0;
    g.act = act;
    g.bn = N > 64 ? 128 : 64;
    g.err = m->d_err;
    return sf_gemm_launch(g, st);
}

// layer C = ELU(A . B^T + bias) [M, N] followed by a linear head of H <= 4 outputs,
// out[r * H + j] = bias_h[j] + sum_c bf16(C[r, c]) wh[j, c], in the GEMM's epilogue
cudaError_t gemm_head(sf_lf* m, cudaStream_t st, const __nv_bfloat16* A, const __nv_bfloat16* B, const float* bias,
                      int M, int N, int K, const __nv_bfloat16* wh, const float* bias_h, int H, float* out) {
    GemmArgs g{};
    g.A = A; g.B = B; g.bias = bias;
    g.M = M; g.N = N; g.Nb = N; g.K = K;
    g.ldc = N; g.ldt = 0;
    g.act = SF_ACT_ELU;
    g.bn = N > 64 ? 128 : 64;
    g.err = m->d_err;
    g.head_w = wh; g.ldhw = N; g.head_b = bias_h; g.head_out = out; g.H = H; g.ldh = H; g.head_act = SF_ACT_NONE;
    return sf_gemm_launch(g, st);
}

}  // namespace

extern "C" {

size_t sf_lf_num_params(void) { return total_params(); }

sf_status sf_lf_create(void* cuda_stream, sf_lf_handle* out) {
    if (!out) return SF_ERR_INVALID_ARG;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SF_ERR_CUDA;
    sf_lf* m = new sf_lf();
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    m->params.assign(total_params(), 0.f);
    bool okk = true;
    for (int g = 0; g < 2; ++g) okk = okk && lalloc(m, &m->img[g], 2 * kImgBytes / 16) && lalloc(m, &m->sb[g], 2 * kHid);
    for (int n = 0; n < 2; ++n)
        for (int t = 0; t < 5; ++t) {
            const int l = t == 0 ? L_EGO0 : t == 1 ? L_EGO1 : t == 2 ? L_TRUNK0 : t == 3 ? L_TRUNK1 : L_HEAD;
            const int o = l == L_HEAD ? (n == 0 ? 3 : 1) : kLayers[l].out;
            const int ip = l == L_EGO0 ? 16 : (kLayers[l].in + 7) / 8 * 8;
            okk = okk && lalloc(m, &m->w[n][t], (size_t)o * ip) && lalloc(m, &m->b[n][t], (size_t)o);
        }
    okk = okk && lalloc(m, &m->d_err, 1);
    okk = okk && cudaStreamCreateWithFlags(&m->aux, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; i < 4 && okk; ++i) okk = cudaEventCreateWithFlags(&m->ev[i], cudaEventDisableTiming) == cudaSuccess;
    static bool attr = false;
    if (okk && !attr) {
        okk = cudaFuncSetAttribute(lf_set_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) ==
                  cudaSuccess &&
              cudaFuncSetAttribute(lf_set_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) ==
                  cudaSuccess;
        attr = okk;
    }
    if (!okk || cudaMemset(m->d_err, 0, 4) != cudaSuccess || upload(m) != SF_OK) {
        for (void* p : m->allocs) cudaFree(p);
        for (cudaEvent_t ev : m->ev)
            if (ev) cudaEventDestroy(ev);
        if (m->aux) cudaStreamDestroy(m->aux);
        delete m;
        return SF_ERR_CUDA;
    }
    *out = m;
    return SF_OK;
}

sf_status sf_lf_destroy(sf_lf_handle m) {
    if (!m) return SF_OK;
    cudaStreamSynchronize(m->stream);
    if (m->aux) cudaStreamSynchronize(m->aux);
    for (cudaEvent_t ev : m->ev)
        if (ev) cudaEventDestroy(ev);
    if (m->aux) cudaStreamDestroy(m->aux);
    for (void* p : m->allocs) cudaFree(p);
    for (void* p : m->acts) cudaFree(p);
    delete m;
    return SF_OK;
}

}  // extern "C"

sf_status sf_lf_reserve(sf_lf_handle m, int batch) { return m ? ensure(m, batch) : SF_ERR_INVALID_ARG; }

extern "C" {

const char* sf_lf_last_error(sf_lf_handle m) { return m ? m->err.c_str() : "NULL handle"; }

sf_status sf_lf_set_params(sf_lf_handle m, const float* h_params, size_t n) {
    if (!m) return SF_ERR_INVALID_ARG;
    if (!h_params || n != total_params())
        return lfail(m, SF_ERR_INVALID_ARG, "sf_lf_set_params: expected " + std::to_string(total_params()) +
                                                " parameters, got " + std::to_string(n));
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(h_params[i])) return lfail(m, SF_ERR_INVALID_ARG, "sf_lf_set_params: non-finite value");
    cudaStreamSynchronize(m->stream);
    m->params.assign(h_params, h_params + n);
    return upload(m);
}

sf_status sf_lf_get_params(sf_lf_handle m, float* h_params, size_t n) {
    if (!m) return SF_ERR_INVALID_ARG;
    if (!h_params || n != total_params()) return lfail(m, SF_ERR_INVALID_ARG, "sf_lf_get_params: wrong size");
    std::memcpy(h_params, m->params.data(), n * 4);
    return SF_OK;
}

}  // extern "C"

sf_status sf_lf_forward_on(sf_lf_handle m, cudaStream_t st, const float* d_obs, const int32_t* d_n_road,
                           const int32_t* d_n_veh, int num_agents, float* d_mean, float* d_value, float* d_embed) {
    if (!m) return SF_ERR_INVALID_ARG;
    if (num_agents < 0 || (num_agents > 0 && (!d_obs || !d_n_road || !d_n_veh || !d_mean)))
        return lfail(m, SF_ERR_INVALID_ARG, "sf_lf_forward: NULL buffer or negative agent count");
    if (num_agents == 0) return SF_OK;
    sf_status s = ensure(m, num_agents);
    if (s != SF_OK) return s;
    const int A = num_agents;
    cudaError_t e = cudaSuccess;
    lf_ego_kernel<<<(A * 16 + 255) / 256, 256, 0, st>>>(d_obs, kObs, A, m->xego);
    e = cudaGetLastError();
    // ego encoders: the actor's on st, the critic's beside it on aux
    if (e == cudaSuccess) e = cudaEventRecord(m->ev[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(m->aux, m->ev[0], 0);
    for (int n = 0; n < 2 && e == cudaSuccess; ++n) {
        cudaStream_t sn = n == 0 ? st : m->aux;
        e = gemm(m, sn, m->xego, m->w[n][0], m->b[n][0], A, 64, 16, SF_ACT_ELU, nullptr, m->he1[n], 64);
        if (e == cudaSuccess) e = gemm(m, sn, m->he1[n], m->w[n][1], m->b[n][1], A, 64, 64, SF_ACT_ELU, nullptr, m->x[n], 256);
    }
    if (e == cudaSuccess) e = cudaEventRecord(m->ev[1], m->aux);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, m->ev[1], 0);
    int sms = 148, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int g = 0; g < 2 && e == cudaSuccess; ++g) {
        SetArgs sa{};
        sa.obs = d_obs; sa.ld = kObs;
        sa.off = g == 0 ? kRoad0 : kVeh0;
        sa.F = g == 0 ? kPT : kNB;
        sa.K = g == 0 ? kKR : kKV;
        sa.count = g == 0 ? d_n_road : d_n_veh;
        sa.num_agents = A;
        sa.wimg = m->img[g];
        sa.b2 = m->sb[g];
        sa.xa = m->x[0]; sa.xc = m->x[1];
        sa.ldx = 256;
        sa.xoff = g == 0 ? 64 : 160;
        sa.err = m->d_err;
        const int items = (A + kG - 1) / kG;
        lf_set_kernel<false><<<2 * (items < sms ? items : sms), kThreads, kSmemBytes, st>>>(sa);
        e = cudaGetLastError();
    }
    // trunks: the actor's on st, the critic's (when the value is wanted) beside it on aux
    if (e == cudaSuccess && d_value) {
        e = cudaEventRecord(m->ev[2], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(m->aux, m->ev[2], 0);
    }
    for (int n = 0; n < 2 && e == cudaSuccess; ++n) {
        if (n == 1 && !d_value) break;   // no value wanted: the critic's trunk is not run
        cudaStream_t sn = n == 0 ? st : m->aux;
        __nv_bfloat16* t1 = n == 0 ? m->t1 : m->t1c;
        e = gemm(m, sn, m->x[n], m->w[n][2], m->b[n][2], A, 128, 256, SF_ACT_ELU, nullptr, t1, 128);
        // trunk layer 2 with the linear head (3 action means, or the value) in its epilogue
        if (e == cudaSuccess)
            e = gemm_head(m, sn, t1, m->w[n][3], m->b[n][3], A, 64, 128, m->w[n][4], m->b[n][4], n == 0 ? 3 : 1,
                          n == 0 ? d_mean : d_value);
    }
    if (e == cudaSuccess && d_value) {
        e = cudaEventRecord(m->ev[3], m->aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, m->ev[3], 0);
    }
    if (e == cudaSuccess && d_embed) {
        lf_embed_kernel<<<(A * 512 + 255) / 256, 256, 0, st>>>(m->x[0], m->x[1], A, d_embed);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return lfail(m, SF_ERR_CUDA, std::string("sf_lf_forward: ") + cudaGetErrorString(e));
    return SF_OK;
}

extern "C" {

sf_status sf_lf_forward(sf_lf_handle m, const float* d_obs, const int32_t* d_n_road, const int32_t* d_n_veh,
                        int num_agents, float* d_mean, float* d_value, float* d_embed) {
    if (!m) return SF_ERR_INVALID_ARG;
    return sf_lf_forward_on(m, m->stream, d_obs, d_n_road, d_n_veh, num_agents, d_mean, d_value, d_embed);
}

sf_status sf_lf_sync(sf_lf_handle m) {
    if (!m) return SF_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return lfail(m, SF_ERR_CUDA, std::string("sf_lf_sync: ") + cudaGetErrorString(e));
    unsigned w = 0;
    if (cudaMemcpy(&w, m->d_err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return lfail(m, SF_ERR_CUDA, "sf_lf_sync");
    if (w) {
        cudaMemset(m->d_err, 0, 4);
        return lfail(m, SF_ERR_TIMEOUT, "sf_lf_sync: a bounded tensor-core wait gave up");
    }
    return SF_OK;
}

}  // extern "C"

// ====================================================================== training
// LfTrainer: the two networks as trainable parts.  Ego encoder: an MLP
// 11 -> 64 -> 64 (ELU, ELU); trunk with its head: an MLP 256 -> 128 -> 64 -> H
// (ELU, ELU, linear); set encoders: fp32 masters updated by Adam, whose bf16
// inference images (the ones the tensor-core set kernel reads) are rebuilt
// after every update, so the training forward and the rollout's forward use
// the same weights.  The trunk input of the training forward is kept in fp32
// (the trunk MLP rounds it to bf16 as the inference path does).

struct LfTrainer {
    sf_lf* lf = nullptr;
    cudaStream_t st = nullptr;
    // the critic's dense MLPs (ego encoder, trunk) run beside the actor's on a second stream
    cudaStream_t aux = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    std::string err;
    std::vector<void*> allocs;
    sf_mlp_handle ego[2] = {nullptr, nullptr}, trunk[2] = {nullptr, nullptr};
    // set encoders: group g's block at goff[g] holds both networks' masters, P[g] floats each
    float *theta = nullptr, *grad = nullptr, *mom = nullptr, *var = nullptr;
    size_t n_set = 0, goff[2] = {0, 0};
    int P[2] = {0, 0};
    // set-encoder backward: per group the distinct-slot counts and first rows of both
    // networks' samples, the row buffers of one (group, network) pass (sized for 96 rows
    // a sample, the most a sample can have) and the split-K partials
    int* nd[2] = {nullptr, nullptr};      // per group [2][cap]
    int* offs[2] = {nullptr, nullptr};    // per group [2][cap + 1]
    BackBufs bb{}, bbv{};                  // road passes (st), vehicle passes (aux; at most 24 rows a sample)
    float *ws1 = nullptr, *ws2 = nullptr, *ws1v = nullptr, *ws2v = nullptr;
    float* sq = nullptr;      // [kSqBlocks]
    int adam_t = 0;
    // batch buffers of the last forward
    int cap = 0, rows = 0;
    float* xf = nullptr;      // [2][cap][256] trunk inputs
    float* dx = nullptr;      // [2][cap][256] their gradients
    float* pmax[2] = {nullptr, nullptr};      // per group [2][cap][96]
    uint16_t* amax[2] = {nullptr, nullptr};
    const float* obs = nullptr;
    const int32_t* cnt[2] = {nullptr, nullptr};
};

namespace {

sf_status tfail(LfTrainer* t, sf_status s, const std::string& msg) {
    if (t) t->err = msg;
    return s;
}

template <class T>
bool talloc(LfTrainer* t, T** p, size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess) return false;
    t->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return cudaMemset(q, 0, count * sizeof(T) + 16) == cudaSuccess;
}

// offsets of every layer's weight and bias in the sf_lf flat layout
struct FlatLayout {
    size_t w[2][9], b[2][9];
};
FlatLayout flat_layout() {
    FlatLayout L{};
    size_t k = 0;
    for (int n = 0; n < 2; ++n)
        for (int l = 0; l < 9; ++l) {
            const int o = l == L_HEAD ? (n == 0 ? 3 : 1) : kLayers[l].out, i = kLayers[l].in;
            L.w[n][l] = k; k += (size_t)o * i;
            L.b[n][l] = k; k += o;
        }
    return L;
}
int layer_out(int n, int l) { return l == L_HEAD ? (n == 0 ? 3 : 1) : kLayers[l].out; }

// (MLP, its layer) of dense layer l of network n
void mlp_of(LfTrainer* t, int n, int l, sf_mlp_handle* m, int* ml) {
    if (l == L_EGO0 || l == L_EGO1) { *m = t->ego[n]; *ml = l - L_EGO0; }
    else { *m = t->trunk[n]; *ml = l - L_TRUNK0; }
}

}  // namespace

sf_status lft_create(sf_lf_handle lf, cudaStream_t st, LfTrainer** out) {
    if (!lf || !out) return SF_ERR_INVALID_ARG;
    *out = nullptr;
    LfTrainer* t = new LfTrainer();
    t->lf = lf;
    t->st = st;
    bool streams_ok = cudaStreamCreateWithFlags(&t->aux, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; i < 2 && streams_ok; ++i)
        streams_ok = cudaEventCreateWithFlags(&t->ev[i], cudaEventDisableTiming) == cudaSuccess;
    if (!streams_ok) {
        lft_destroy(t);
        return SF_ERR_CUDA;
    }
    const FlatLayout FL = flat_layout();
    const float* P = lf->params.data();
    bool ok = true;
    for (int n = 0; n < 2 && ok; ++n) {
        const int de[3] = {kLayers[L_EGO0].in, kLayers[L_EGO0].out, kLayers[L_EGO1].out};
        const int dt[4] = {kLayers[L_TRUNK0].in, kLayers[L_TRUNK0].out, kLayers[L_TRUNK1].out, n == 0 ? 3 : 1};
        ok = sf_mlp_create(2, de, SF_ACT_ELU, SF_ACT_ELU, st, &t->ego[n]) == SF_OK &&
             sf_mlp_create(3, dt, SF_ACT_ELU, SF_ACT_NONE, st, &t->trunk[n]) == SF_OK;
        for (int l : {L_EGO0, L_EGO1, L_TRUNK0, L_TRUNK1, L_HEAD}) {
            if (!ok) break;
            sf_mlp_handle m;
            int ml;
            mlp_of(t, n, l, &m, &ml);
            ok = sf_mlp_set_layer(m, ml, P + FL.w[n][l], P + FL.b[n][l]) == SF_OK;
        }
    }
    for (int g = 0; g < 2; ++g) {
        const int F = g == 0 ? kPT : kNB;
        t->P[g] = kHid * F + kHid + kHid * kHid + kHid;
    }
    t->goff[1] = 2 * (size_t)t->P[0];
    t->n_set = 2 * (size_t)(t->P[0] + t->P[1]);
    ok = ok && talloc(t, &t->theta, t->n_set) && talloc(t, &t->grad, t->n_set) && talloc(t, &t->mom, t->n_set) &&
         talloc(t, &t->var, t->n_set) && talloc(t, &t->sq, kSqBlocks) &&
         talloc(t, &t->ws1, (size_t)kBackSplit * kHid * 16) && talloc(t, &t->ws2, (size_t)kBackSplit * kHid * kLdW2) &&
         talloc(t, &t->ws1v, (size_t)kBackSplit * kHid * 16) && talloc(t, &t->ws2v, (size_t)kBackSplit * kHid * kLdW2) &&
         talloc(t, &t->bb.w1b, (size_t)kHid * 16) && talloc(t, &t->bb.w2t, (size_t)kHid * kHid) &&
         talloc(t, &t->bbv.w1b, (size_t)kHid * 16) && talloc(t, &t->bbv.w2t, (size_t)kHid * kHid);
    if (ok) {   // the masters from the network's parameters: group blocks are contiguous in the flat layout
        std::vector<float> h(t->n_set);
        for (int g = 0; g < 2; ++g)
            for (int n = 0; n < 2; ++n) {
                const int l0 = g == 0 ? L_ROAD0 : L_VEH0;
                std::memcpy(h.data() + t->goff[g] + (size_t)n * t->P[g], P + FL.w[n][l0], (size_t)t->P[g] * 4);
            }
        ok = cudaMemcpy(t->theta, h.data(), t->n_set * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (!ok) {
        lft_destroy(t);
        return SF_ERR_OOM;
    }
    *out = t;
    return SF_OK;
}

void lft_destroy(LfTrainer* t) {
    if (!t) return;
    cudaStreamSynchronize(t->st);
    if (t->aux) cudaStreamSynchronize(t->aux);
    for (cudaEvent_t ev : t->ev)
        if (ev) cudaEventDestroy(ev);
    if (t->aux) cudaStreamDestroy(t->aux);
    for (int n = 0; n < 2; ++n) {
        sf_mlp_destroy(t->ego[n]);
        sf_mlp_destroy(t->trunk[n]);
    }
    for (void* p : t->allocs) cudaFree(p);
    delete t;
}

const char* lft_error(LfTrainer* t) { return t ? t->err.c_str() : "NULL trainer"; }

namespace {
// fork the second stream from st (false: a CUDA error)
bool lft_fork(LfTrainer* t) {
    return cudaEventRecord(t->ev[0], t->st) == cudaSuccess && cudaStreamWaitEvent(t->aux, t->ev[0], 0) == cudaSuccess;
}
bool lft_join(LfTrainer* t) {
    return cudaEventRecord(t->ev[1], t->aux) == cudaSuccess && cudaStreamWaitEvent(t->st, t->ev[1], 0) == cudaSuccess;
}
sf_status lft_reserve(LfTrainer* t, int rows) {
    if (rows <= t->cap) return SF_OK;
    cudaStreamSynchronize(t->st);
    bool ok = talloc(t, &t->xf, (size_t)2 * rows * 256) && talloc(t, &t->dx, (size_t)2 * rows * 256);
    for (int g = 0; g < 2 && ok; ++g)
        ok = talloc(t, &t->pmax[g], (size_t)2 * rows * kHid) && talloc(t, &t->amax[g], (size_t)2 * rows * kHid) &&
             talloc(t, &t->nd[g], (size_t)2 * rows) && talloc(t, &t->offs[g], (size_t)2 * (rows + 1));
    // the backward's rows: at most 96 a sample (one per pooled feature) on the road group, 24 (its
    // slots) on the vehicle group
    for (int g = 0; g < 2 && ok; ++g) {
        const size_t per = g == 0 ? kHid : kKV;
        const size_t ldcap = std::max<size_t>(128, (per * rows + 63) / 64 * 64);
        BackBufs& o = g == 0 ? t->bb : t->bbv;
        ok = talloc(t, &o.x, ldcap * 16) && talloc(t, &o.xt, 16 * ldcap) && talloc(t, &o.dz2, ldcap * kHid) &&
             talloc(t, &o.dz2t, kHid * ldcap) && talloc(t, &o.h1t, (kHid + 1) * ldcap) &&
             talloc(t, &o.dh1t, kHid * ldcap) && talloc(t, &o.dz1t, kHid * ldcap);
    }
    for (int n = 0; n < 2 && ok; ++n)
        ok = sf_mlp_reserve(t->ego[n], rows) == SF_OK && sf_mlp_reserve(t->trunk[n], rows) == SF_OK;
    if (!ok) return tfail(t, SF_ERR_OOM, "late-fusion training buffers");
    t->cap = rows;   // buffers of a smaller batch stay allocated until destroy
    return SF_OK;
}
}  // namespace

sf_status lft_forward(LfTrainer* t, const float* d_obs, const int32_t* d_n_road, const int32_t* d_n_veh, int rows,
                      float* d_mean, float* d_value) {
    if (!t || !d_obs || !d_n_road || !d_n_veh || !d_mean || !d_value || rows < 8 || rows % 8)
        return SF_ERR_INVALID_ARG;
    sf_status s = lft_reserve(t, rows);
    if (s != SF_OK) return s;
    const size_t xnet = (size_t)rows * 256;
    t->rows = rows;
    t->obs = d_obs;
    t->cnt[0] = d_n_road;
    t->cnt[1] = d_n_veh;
    if (!lft_fork(t)) return tfail(t, SF_ERR_CUDA, "late-fusion training forward: stream fork");
    for (int n = 0; n < 2 && s == SF_OK; ++n)   // ego encoders into trunk-input columns 0..63 (the critic's on aux)
        s = sf_mlp_forward_train_on(t->ego[n], n == 0 ? t->st : t->aux, d_obs, kObs, rows, t->xf + n * xnet, 256);
    if (!lft_join(t) && s == SF_OK) s = SF_ERR_CUDA;
    if (s != SF_OK) return tfail(t, s, "late-fusion training forward: ego encoder");
    int sms = 148, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaSuccess;
    for (int g = 0; g < 2 && e == cudaSuccess; ++g) {
        SetArgs sa{};
        sa.obs = d_obs; sa.ld = kObs;
        sa.off = g == 0 ? kRoad0 : kVeh0;
        sa.F = g == 0 ? kPT : kNB;
        sa.K = g == 0 ? kKR : kKV;
        sa.count = t->cnt[g];
        sa.num_agents = rows;
        sa.wimg = t->lf->img[g];
        sa.b2 = t->lf->sb[g];
        sa.xa = nullptr; sa.xc = nullptr; sa.ldx = 256;
        sa.xoff = g == 0 ? 64 : 160;
        sa.err = t->lf->d_err;
        sa.xf = t->xf; sa.xf_net = xnet; sa.ldxf = 256;
        sa.pmax = t->pmax[g]; sa.amax = t->amax[g];
        const int items = (rows + kGTrain - 1) / kGTrain;
        lf_set_kernel<true><<<2 * (items < sms ? items : sms), kThreads, kSmemBytes, t->st>>>(sa);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return tfail(t, SF_ERR_CUDA, std::string("late-fusion training forward: ") + cudaGetErrorString(e));
    if (!lft_fork(t)) return tfail(t, SF_ERR_CUDA, "late-fusion training forward: stream fork");
    s = sf_mlp_forward_train_on(t->trunk[0], t->st, t->xf, 256, rows, d_mean, 3);
    if (s == SF_OK) s = sf_mlp_forward_train_on(t->trunk[1], t->aux, t->xf + xnet, 256, rows, d_value, 1);
    if (!lft_join(t) && s == SF_OK) s = SF_ERR_CUDA;
    return s == SF_OK ? SF_OK : tfail(t, s, "late-fusion training forward: trunk");
}

namespace {
// one product of the set-encoder backward on the tensor cores: C = A B^T (A [M][K], B [N][K]
// bf16), written transposed (out_t [N][ldt]) or as split-K partials (ws [splits][M][ldc])
cudaError_t back_gemm(LfTrainer* t, cudaStream_t st, const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N,
                      int K, int act, __nv_bfloat16* out_t, int ldt, float* ws, int splits, int ldc, int bn) {
    GemmArgs g{};
    g.A = A; g.B = B; g.M = M; g.N = N; g.Nb = N; g.K = K; g.act = act;
    g.out_bf16_t = out_t; g.ldt = ldt;
    g.ws = ws; g.splits = splits; g.ldc = ldc;
    g.bn = bn;
    g.err = t->lf->d_err;
    return sf_gemm_launch(g, st);
}
}  // namespace

sf_status lft_backward(LfTrainer* t, const float* d_dmean, const float* d_dvalue, int rows) {
    if (!t || !d_dmean || !d_dvalue || rows != t->rows) return SF_ERR_INVALID_ARG;
    const size_t xnet = (size_t)rows * 256;
    // each network's trunk then ego encoder, the critic's on aux
    if (!lft_fork(t)) return tfail(t, SF_ERR_CUDA, "late-fusion backward: stream fork");
    sf_status s = sf_mlp_backward_dx_on(t->trunk[0], t->st, d_dmean, 3, rows, t->dx, 256);
    if (s == SF_OK) s = sf_mlp_backward_on(t->ego[0], t->st, t->dx, 256, rows);
    if (s == SF_OK) s = sf_mlp_backward_dx_on(t->trunk[1], t->aux, d_dvalue, 1, rows, t->dx + xnet, 256);
    if (s == SF_OK) s = sf_mlp_backward_on(t->ego[1], t->aux, t->dx + xnet, 256, rows);
    if (!lft_join(t) && s == SF_OK) s = SF_ERR_CUDA;
    if (s != SF_OK) return tfail(t, s, "late-fusion backward: dense layers");
    // set encoders: the rows of every (group, network) pass, counted first (one wait for
    // the four row totals, which size the products), then the products pass by pass
    cudaError_t e = cudaSuccess;
    BackRows br[2];
    int tot[2][2] = {{0, 0}, {0, 0}};
    for (int g = 0; g < 2 && e == cudaSuccess; ++g) {
        BackRows& b = br[g];
        b = BackRows{};
        b.obs = t->obs; b.ld = kObs;
        b.off = g == 0 ? kRoad0 : kVeh0;
        b.F = g == 0 ? kPT : kNB;
        b.K = g == 0 ? kKR : kKV;
        b.count = t->cnt[g];
        b.B = rows;
        b.theta = t->theta + t->goff[g];
        b.theta_net = t->P[g];
        b.pmax = t->pmax[g];
        b.amax = t->amax[g];
        b.dx = t->dx; b.dx_net = xnet; b.lddx = 256;
        b.xoff = g == 0 ? 64 : 160;
        b.nd = t->nd[g];
        b.offs = t->offs[g];
        lfb_count_kernel<<<dim3((unsigned)((rows + 7) / 8), 2), 256, 0, t->st>>>(b);
        lfb_scan_kernel<<<2, 1024, 0, t->st>>>(b.nd, rows, b.offs);
        e = cudaGetLastError();
        for (int n = 0; n < 2 && e == cudaSuccess; ++n)
            e = cudaMemcpyAsync(&tot[g][n], b.offs + (size_t)n * (rows + 1) + rows, sizeof(int), cudaMemcpyDeviceToHost,
                                t->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(t->st);
    // the road passes on st, the vehicle passes beside them on aux (buffers of their own)
    if (e == cudaSuccess && !lft_fork(t)) e = cudaErrorUnknown;
    for (int g = 0; g < 2 && e == cudaSuccess; ++g)
        for (int n = 0; n < 2 && e == cudaSuccess; ++n) {
            const int R = tot[g][n], F = br[g].F, P = t->P[g];
            cudaStream_t sg = g == 0 ? t->st : t->aux;
            float* ws1 = g == 0 ? t->ws1 : t->ws1v;
            float* ws2 = g == 0 ? t->ws2 : t->ws2v;
            float* gout = t->grad + t->goff[g] + (size_t)n * P;
            if (R <= 0) {   // no sample of this group has a filled slot: no gradient
                e = cudaMemsetAsync(gout, 0, (size_t)P * 4, sg);
                continue;
            }
            BackBufs o = g == 0 ? t->bb : t->bbv;
            o.ldR = std::max(128, (R + 63) / 64 * 64);
            const int S = std::min(kBackSplit, o.ldR / 64);   // the GEMM's split of ldR / 64 K tiles
            lfb_weights_kernel<<<(kHid * 16 + kHid * kHid + 255) / 256, 256, 0, sg>>>(
                br[g].theta + (size_t)n * P, F, o.w1b, o.w2t);
            lfb_rows_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, sg>>>(br[g], o, n);
            lfb_pad_kernel<<<16 + kHid + 1, 128, 0, sg>>>(o, R);
            e = cudaGetLastError();
            // dH1^T = (dZ2 W2)^T on the tensor cores; H1^T and dZ1^T
            if (e == cudaSuccess)
                e = back_gemm(t, sg, o.dz2, o.w2t, R, kHid, kHid, SF_ACT_NONE, o.dh1t, o.ldR, nullptr, 1, kHid, 128);
            if (e == cudaSuccess) {
                lfb_h1dz1_kernel<<<(unsigned)((o.ldR / 2 + 255) / 256), 256, 0, sg>>>(o, R);
                e = cudaGetLastError();
            }
            // [dW2 | db2] = dZ2^T [H1 | 1]; [dW1 | . | db1] = dZ1^T X (K: the rows, split)
            if (e == cudaSuccess)
                e = back_gemm(t, sg, o.dz2t, o.h1t, kHid, kHid + 1, o.ldR, SF_ACT_NONE, nullptr, 0, ws2, S, kLdW2, 128);
            if (e == cudaSuccess)
                e = back_gemm(t, sg, o.dz1t, o.xt, kHid, 16, o.ldR, SF_ACT_NONE, nullptr, 0, ws1, S, 16, 64);
            if (e == cudaSuccess) {
                lfb_reduce_kernel<<<(unsigned)((P + 255) / 256), 256, 0, sg>>>(ws1, S, ws2, S, F, gout);
                e = cudaGetLastError();
            }
        }
    if (e == cudaSuccess && !lft_join(t)) e = cudaErrorUnknown;
    return e == cudaSuccess ? SF_OK
                            : tfail(t, SF_ERR_CUDA, std::string("late-fusion backward: ") + cudaGetErrorString(e));
}

sf_status lft_grad_sumsq(LfTrainer* t, float* d_acc) {
    if (!t || !d_acc) return SF_ERR_INVALID_ARG;
    sf_status s = SF_OK;
    for (int n = 0; n < 2 && s == SF_OK; ++n) {
        s = sf_mlp_grad_sumsq_on(t->ego[n], t->st, d_acc);
        if (s == SF_OK) s = sf_mlp_grad_sumsq_on(t->trunk[n], t->st, d_acc);
    }
    if (s != SF_OK) return tfail(t, s, "late-fusion gradient norm");
    lf_sumsq_part_kernel<<<kSqBlocks, 256, 0, t->st>>>(t->grad, t->n_set, t->sq);
    lf_sumsq_final_kernel<<<1, 32, 0, t->st>>>(t->sq, kSqBlocks, d_acc);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SF_OK : tfail(t, SF_ERR_CUDA, cudaGetErrorString(e));
}

sf_status lft_adam(LfTrainer* t, const float* d_lr, const float* d_scale) {
    if (!t || !d_lr || !d_scale) return SF_ERR_INVALID_ARG;
    sf_status s = SF_OK;
    for (int n = 0; n < 2 && s == SF_OK; ++n) {
        s = sf_mlp_adam_on(t->ego[n], t->st, d_lr, d_scale);
        if (s == SF_OK) s = sf_mlp_adam_on(t->trunk[n], t->st, d_lr, d_scale);
    }
    if (s != SF_OK) return tfail(t, s, "late-fusion Adam");
    ++t->adam_t;
    const float c1 = 1.f - std::pow(0.9f, (float)t->adam_t), c2 = 1.f - std::pow(0.999f, (float)t->adam_t);
    lf_adam_kernel<<<(unsigned)((t->n_set + 255) / 256), 256, 0, t->st>>>(t->theta, t->grad, t->mom, t->var, t->n_set,
                                                                          d_lr, d_scale, c1, c2);
    for (int g = 0; g < 2; ++g) {   // the tensor-core set kernel's images follow the masters
        const int per = kHid * 16 + kHid * kHid + kHid;
        lf_image_kernel<<<(unsigned)((2 * per + 255) / 256), 256, 0, t->st>>>(
            t->theta + t->goff[g], t->P[g], g == 0 ? kPT : kNB, reinterpret_cast<unsigned char*>(t->lf->img[g]),
            t->lf->sb[g]);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SF_OK : tfail(t, SF_ERR_CUDA, cudaGetErrorString(e));
}

sf_status lft_publish(LfTrainer* t) {
    if (!t) return SF_ERR_INVALID_ARG;
    const int dl[5] = {L_EGO0, L_EGO1, L_TRUNK0, L_TRUNK1, L_HEAD};
    cudaError_t e = cudaSuccess;
    for (int n = 0; n < 2 && e == cudaSuccess; ++n)
        for (int k = 0; k < 5 && e == cudaSuccess; ++k) {
            sf_mlp_handle m;
            int ml, ld = 0;
            mlp_of(t, n, dl[k], &m, &ml);
            const void* wb = nullptr;
            const float* b = nullptr;
            if (sf_mlp_device_layer(m, ml, &wb, &ld, &b) != SF_OK) return tfail(t, SF_ERR_STATE, "layer pointers");
            const int o = layer_out(n, dl[k]);
            // the same [out][in padded] bf16 layout as the inference network's (ego input padded to 16)
            e = cudaMemcpyAsync(t->lf->w[n][k], wb, (size_t)o * ld * 2, cudaMemcpyDeviceToDevice, t->st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(t->lf->b[n][k], b, (size_t)o * 4, cudaMemcpyDeviceToDevice, t->st);
        }
    return e == cudaSuccess ? SF_OK : tfail(t, SF_ERR_CUDA, std::string("publish: ") + cudaGetErrorString(e));
}

sf_status lft_argmax(LfTrainer* t, uint16_t* d_out) {
    if (!t || !d_out || t->rows <= 0) return SF_ERR_INVALID_ARG;
    const size_t n = (size_t)2 * t->rows * kHid;
    cudaError_t e = cudaMemcpyAsync(d_out, t->amax[0], n * 2, cudaMemcpyDeviceToDevice, t->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_out + n, t->amax[1], n * 2, cudaMemcpyDeviceToDevice, t->st);
    return e == cudaSuccess ? SF_OK : tfail(t, SF_ERR_CUDA, cudaGetErrorString(e));
}

sf_status lft_get(LfTrainer* t, float* h_params, float* h_grads) {
    if (!t || (!h_params && !h_grads)) return SF_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(t->st) != cudaSuccess) return tfail(t, SF_ERR_CUDA, "synchronize");
    const FlatLayout FL = flat_layout();
    for (int n = 0; n < 2; ++n)
        for (int l : {L_EGO0, L_EGO1, L_TRUNK0, L_TRUNK1, L_HEAD}) {
            sf_mlp_handle m;
            int ml;
            mlp_of(t, n, l, &m, &ml);
            const sf_status s = sf_mlp_get_layer(m, ml, h_params ? h_params + FL.w[n][l] : nullptr,
                                                 h_params ? h_params + FL.b[n][l] : nullptr,
                                                 h_grads ? h_grads + FL.w[n][l] : nullptr,
                                                 h_grads ? h_grads + FL.b[n][l] : nullptr);
            if (s != SF_OK) return tfail(t, s, "dense layer read-back");
        }
    std::vector<float> hp(t->n_set), hg(t->n_set);
    if (cudaMemcpy(hp.data(), t->theta, t->n_set * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(hg.data(), t->grad, t->n_set * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return tfail(t, SF_ERR_CUDA, "set encoder read-back");
    for (int g = 0; g < 2; ++g)
        for (int n = 0; n < 2; ++n) {
            const int l0 = g == 0 ? L_ROAD0 : L_VEH0;
            const size_t src = t->goff[g] + (size_t)n * t->P[g];
            if (h_params) std::memcpy(h_params + FL.w[n][l0], hp.data() + src, (size_t)t->P[g] * 4);
            if (h_grads) std::memcpy(h_grads + FL.w[n][l0], hg.data() + src, (size_t)t->P[g] * 4);
        }
    return SF_OK;
}
