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
constexpr uint32_t kTmemCols = 256;                 // D1 at column 0 (96), D2 at column 128 (128)

struct SetArgs {
    const float* obs;          // [A][ld]
    int ld, off, F, K;         // row stride, group offset, features per slot, slots
    const int32_t* count;      // [A] filled slots
    int num_agents;
    const uint4* wimg;         // 2 x kImgBytes: actor then critic weight images (bf16, swizzled)
    const float* b2;           // [2][96] layer-2 biases (layer-1 biases are in the images)
    __nv_bfloat16* xa;         // [A][ldx] actor trunk input
    __nv_bfloat16* xc;         // [A][ldx] critic trunk input
    int ldx, xoff;             // columns [xoff, xoff + 96) receive the pooled embedding
    unsigned* err;
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

// ELU of two fp32 accumulators, in packed bf16: the positive part is the
// rounded input, the negative part 2^(x log2 e) - 1 from the two-lane bf16
// exp2; one of the two parts is zero, so their sum is exact
__device__ __forceinline__ uint32_t elu_bf16x2(uint32_t a, uint32_t b) {
    uint32_t x, pos, neg, e, t, y;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(x) : "f"(__uint_as_float(b)), "f"(__uint_as_float(a)));
    asm("max.bf16x2 %0, %1, %2;" : "=r"(pos) : "r"(x), "r"(0u));
    asm("min.bf16x2 %0, %1, %2;" : "=r"(neg) : "r"(x), "r"(0u));
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(neg) : "r"(neg), "r"(0x3FB93FB9u));   // log2(e) in bf16
    asm("ex2.approx.ftz.bf16x2 %0, %1;" : "=r"(e) : "r"(neg));
    asm("sub.rn.bf16x2 %0, %1, %2;" : "=r"(t) : "r"(e), "r"(0x3F803F80u));       // e - 1 (exact for e >= 1/2)
    asm("add.rn.bf16x2 %0, %1, %2;" : "=r"(y) : "r"(pos), "r"(t));
    return y;
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
__global__ void __launch_bounds__(kThreads, 2) lf_set_kernel(const SetArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(sm);
    uint32_t* pool = reinterpret_cast<uint32_t*>(sm + kOffPool);
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
    for (int i = tid; i < kG * kHid; i += kThreads) pool[i] = 0u;
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
    const int num_items = (a.num_agents + kG - 1) / kG;

    for (int item = cta; item < num_items && ok; item += ncta) {
        const int a0 = item * kG;
        const int na = min(kG, a.num_agents - a0);
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
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int s = (int)((md[i] >> 8) & 0xFFu), valid = (int)(md[i] & 0xFFu);
                    if (s != cur) {                      // warp-uniform: the group starts the next agent
                        if (cur >= 0 && cur < kG) atomicMax(&pool[cur * kHid + f], fkey(m));
                        cur = s;
                        m = -INFINITY;
                    }
                    if (s >= kG) continue;               // rows past the item
                    const uint32_t* v = r[i >> 2] + 8 * (i & 3);
                    float x[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) x[k] = __uint_as_float(v[k]);
                    if (valid < 8) {                     // warp-uniform: the agent's last, partly filled group
#pragma unroll
                        for (int k = 1; k < 8; ++k) x[k] = k < valid ? x[k] : x[0];
                    }
                    m = max3f(max3f(m, x[0], x[1]), max3f(x[2], x[3], x[4]), max3f(x[5], x[6], x[7]));
                }
                if (cur >= 0 && cur < kG) atomicMax(&pool[cur * kHid + f], fkey(m));   // continues past these rows
            }
            tc_before();   // this tile's TMEM reads before the next tile's barrier and MMAs
        }
        if (!ok) break;
        __syncthreads();
        if (*abort_flag) break;
        // ---- the item's pooled embeddings: + bias, ELU, bf16 into the trunk inputs
        for (int i = tid; i < na * kHid; i += kThreads) {
            const int al = i / kHid, col = i - al * kHid;
            const uint32_t k = pool[i];
            pool[i] = 0u;
            const float y = k ? elu(funkey(k) + sb2[col]) : 0.f;
            X[(size_t)(a0 + al) * a.ldx + a.xoff + col] = __float2bfloat16_rn(y);
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
    __nv_bfloat16 *t1 = nullptr, *t2 = nullptr;
    unsigned* d_err = nullptr;
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
               lalloc(m, &m->t2, Aa * 64, true);
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
    static bool attr = false;
    if (okk && !attr) {
        okk = cudaFuncSetAttribute(lf_set_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) ==
              cudaSuccess;
        attr = okk;
    }
    if (!okk || cudaMemset(m->d_err, 0, 4) != cudaSuccess || upload(m) != SF_OK) {
        for (void* p : m->allocs) cudaFree(p);
        delete m;
        return SF_ERR_CUDA;
    }
    *out = m;
    return SF_OK;
}

sf_status sf_lf_destroy(sf_lf_handle m) {
    if (!m) return SF_OK;
    cudaStreamSynchronize(m->stream);
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
    for (int n = 0; n < 2 && e == cudaSuccess; ++n) {
        e = gemm(m, st, m->xego, m->w[n][0], m->b[n][0], A, 64, 16, SF_ACT_ELU, nullptr, m->he1[n], 64);
        if (e == cudaSuccess) e = gemm(m, st, m->he1[n], m->w[n][1], m->b[n][1], A, 64, 64, SF_ACT_ELU, nullptr, m->x[n], 256);
    }
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
        lf_set_kernel<<<2 * (items < sms ? items : sms), kThreads, kSmemBytes, st>>>(sa);
        e = cudaGetLastError();
    }
    for (int n = 0; n < 2 && e == cudaSuccess; ++n) {
        if (n == 1 && !d_value) break;   // no value wanted: the critic's trunk is not run
        e = gemm(m, st, m->x[n], m->w[n][2], m->b[n][2], A, 128, 256, SF_ACT_ELU, nullptr, m->t1, 128);
        // trunk layer 2 with the linear head (3 action means, or the value) in its epilogue
        if (e == cudaSuccess)
            e = gemm_head(m, st, m->t1, m->w[n][3], m->b[n][3], A, 64, 128, m->w[n][4], m->b[n][4], n == 0 ? 3 : 1,
                          n == 0 ? d_mean : d_value);
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
