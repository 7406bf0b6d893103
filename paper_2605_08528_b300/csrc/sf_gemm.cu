// sf_gemm.cu -- persistent BF16 tensor-core GEMM with a fused epilogue for the MLPs (sm_103a).
//
//   C[M, N] = act(A[M, K] . B[N, K]^T + bias[N])
//
// A and B are bf16, row-major with K contiguous (B is a weight matrix stored
// [out, in]); accumulation is fp32.  One persistent CTA per SM walks a static
// list of work units (CTA c takes units c, c + grid, ...): a unit is one
// 128 x BN output tile, or, with a fused head, every column tile of one
// 128-row block.  Fourteen warps:
//   warp 0 lane 0  TMA producer: 128 x 64 (A) and BN x 64 (B) K-tiles into a
//                  kStages-deep ring (128-byte swizzle), running ahead across
//                  tile boundaries;
//   warp 1 lane 0  MMA issuer: tcgen05.mma (M 128, N BN, K 16) into one of two
//                  TMEM accumulators of BN fp32 columns, alternating per tile,
//                  so that the MMAs of tile i + 1 run while tile i is drained;
//   warps 2-13     epilogue: tcgen05.ld of a finished accumulator (warp w reads
//                  TMEM lanes 32(w % 4)..+31 and every third 32-column chunk,
//                  starting at chunk (w - 2) / 4), bias, activation, stores
//                  staged through shared memory so that they coalesce, and the
//                  optional narrow head; then release of the accumulator to the
//                  MMA issuer.  Three warps per lane slice hide more of the
//                  latency of the TMEM loads and the exponentials than two, and
//                  fourteen warps in all still leave 128 registers a thread.
// Every mbarrier wait is bounded: on expiry the kernel records SF_GEMM_TIMEOUT
// in the error word and raises an abort flag that every role polls, so all of
// them stop issuing; before it frees its TMEM and returns, the CTA waits
// (bounded, 1 s) for every MMA and every TMA load it issued, so no
// asynchronous operation outlives it.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "sf_gemm.cuh"
#include "sf_tc.cuh"

namespace {

constexpr int kBM = 128, kBK = 64;
constexpr int kParts = 3;            // epilogue warps per TMEM lane slice, each every third column chunk
constexpr int kEpiWarps = 4 * kParts;
constexpr int kThreads = 64 + 32 * kEpiWarps;   // producer warp, MMA warp, epilogue warps
constexpr int kMaxHead = 4;
constexpr int kHeadMaxN = 512;       // widest layer a head can follow
constexpr int kBiasSmemN = 512;      // biases of layers up to this width are read from shared memory
// ring depth: 192 KB of operand stages at every tile width, enough bytes in
// flight to cover the L2 latency at the tensor cores' rate
template <int BN>
constexpr int stages_for() { return BN >= 256 ? 4 : (BN >= 128 ? 6 : 8); }
using namespace sftc;

// bounded wait that also gives up when another role has raised the abort flag;
// on its own expiry it records the timeout and raises the flag
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile uint32_t* abort,
                                              unsigned* err, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 63) {
            if (*abort) return false;
            if (global_ns() - t0 > limit_ns) break;
        }
    }
    if (err) atomicOr(err, SF_GEMM_TIMEOUT);
    *abort = 1;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 32 rows x 64 bytes (lane = row, w = the row's four 16-byte pieces) stored through
// the warp's 1 KB staging buffer, 16 rows at a time, so that every store
// instruction writes 8 rows of 64 contiguous bytes; the staged piece c of row r
// sits at r * 64 + ((c ^ ((r >> 1) & 3)) * 16), which keeps both the row-wise
// writes and the column-wise reads free of bank conflicts.  Rows at or beyond
// rows_valid are not stored.
__device__ __forceinline__ void stage_store(unsigned char* stg, const uint4 (&w)[4], unsigned char* g,
                                            size_t ld_bytes, int rows_valid, int lane) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if ((lane >> 4) == h) {
            const int rr = lane & 15;
#pragma unroll
            for (int c = 0; c < 4; ++c) *reinterpret_cast<uint4*>(stg + rr * 64 + ((c ^ ((rr >> 1) & 3)) << 4)) = w[c];
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int rr = i * 8 + (lane >> 2), c = lane & 3, row = 16 * h + rr;
            const uint4 x = *reinterpret_cast<const uint4*>(stg + rr * 64 + ((c ^ ((rr >> 1) & 3)) << 4));
            if (row < rows_valid) *reinterpret_cast<uint4*>(g + row * ld_bytes + c * 16) = x;
        }
        __syncwarp();
    }
}

// 32 fp32 values of each of the warp's 32 rows, columns [0, 32) from g, as two 64-byte halves
__device__ __forceinline__ void stage_store_f32(unsigned char* stg, const float (&v)[32], float* g, size_t ld,
                                                int rows_valid, int lane) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint4 w[4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
            w[c] = make_uint4(__float_as_uint(v[16 * h + 4 * c]), __float_as_uint(v[16 * h + 4 * c + 1]),
                              __float_as_uint(v[16 * h + 4 * c + 2]), __float_as_uint(v[16 * h + 4 * c + 3]));
        stage_store(stg, w, reinterpret_cast<unsigned char*>(g + 16 * h), ld * 4, rows_valid, lane);
    }
}

// the same for 32 bf16 values (round to nearest) per row
__device__ __forceinline__ void stage_store_bf16(unsigned char* stg, const float (&v)[32], __nv_bfloat16* g,
                                                 size_t ld, int rows_valid, int lane) {
    uint4 w[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t p[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * c + 2 * e], v[8 * c + 2 * e + 1]);
            p[e] = *reinterpret_cast<const uint32_t*>(&h2);
        }
        w[c] = make_uint4(p[0], p[1], p[2], p[3]);
    }
    stage_store(stg, w, reinterpret_cast<unsigned char*>(g), ld * 2, rows_valid, lane);
}

// activations of 32 accumulator values; the exponentials use the hardware
// exp2-based intrinsic (relative error far below the bf16 output rounding)
__device__ __forceinline__ void activate32(float (&v)[32], int act) {
    if (act == SF_ACT_ELU) {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = v[i] > 0.f ? v[i] : __expf(v[i]) - 1.f;
    } else if (act == SF_ACT_SILU) {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = __fdividef(v[i], 1.f + __expf(-v[i]));
    } else if (act == SF_ACT_TANH) {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = tanhf(v[i]);
    }
}

__device__ __forceinline__ float activate1(float v, int act) {
    if (act == SF_ACT_ELU) return v > 0.f ? v : __expf(v) - 1.f;
    if (act == SF_ACT_SILU) return __fdividef(v, 1.f + __expf(-v));
    if (act == SF_ACT_TANH) return tanhf(v);
    return v;
}

template <int BN, int kStages>
struct alignas(1024) GemmSmem {
    __nv_bfloat16 a[kStages][kBM * kBK];
    __nv_bfloat16 b[kStages][BN * kBK];
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t acc_full[2];     // MMA issuer -> epilogue: accumulator b holds a finished tile
    uint64_t acc_empty[2];    // epilogue (every warp) -> MMA issuer: accumulator b was read
    uint64_t head_full[2];    // column parts 1.. (kParts - 1) x 128 threads -> part 0: head partials written
    uint64_t done;
    // per epilogue warp: 16 rows x 64 B for coalesced stores (16-byte vector accesses)
    alignas(128) unsigned char stage[kEpiWarps][16 * 64];
    alignas(16) float hw[kMaxHead][kHeadMaxN];   // head weights (bf16 values as fp32; zero beyond N)
    alignas(16) float bias[kBiasSmemN];          // the layer's bias when N <= kBiasSmemN
    float head[2][kParts - 1][kBM][kMaxHead];   // column parts 1..: head partial sums, by unit parity
    uint32_t tmem_base;
    uint32_t abort;           // a wait gave up: every role stops issuing
    int issued;               // K tiles whose TMA loads the producer issued
};

template <int BN, int kStages>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                   const GemmArgs args) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    GemmSmem<BN, kStages>& S = *reinterpret_cast<GemmSmem<BN, kStages>*>(
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (args.K + kBK - 1) / kBK;
    const int mt = (args.M + kBM - 1) / kBM, nt = (args.N + BN - 1) / BN;
    const bool headed = args.head_w != nullptr;
    const int nsplit = args.ws ? args.splits : 1;
    // work units: with a head, unit u is row block u with its nt column tiles; else one tile
    const int units = headed ? mt : mt * nt * nsplit, per_unit = headed ? nt : 1;
    volatile uint32_t* abort = &S.abort;
    const uint64_t lim = args.wait_ns ? args.wait_ns : kWaitNs;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) { mbar_init(&S.full[s], 1); mbar_init(&S.empty[s], 1); }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&S.acc_full[b], 1);
            mbar_init(&S.acc_empty[b], kEpiWarps);
            mbar_init(&S.head_full[b], (kParts - 1) * kBM);
        }
        mbar_init(&S.done, 1);
        S.abort = 0;
        S.issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (headed)   // the head weights as fp32, zero beyond N (columns past N then add nothing)
        for (int e = threadIdx.x; e < kMaxHead * kHeadMaxN; e += kThreads) {
            const int j = e / kHeadMaxN, c = e - j * kHeadMaxN;
            S.hw[j][c] = (j < args.H && c < args.N) ? __bfloat162float(args.head_w[(size_t)j * args.ldhw + c]) : 0.f;
        }
    const bool bias_smem = args.bias && args.N <= kBiasSmemN;
    if (bias_smem)   // every tile's epilogue reads the bias: one copy per CTA, read at shared-memory latency
        for (int e = threadIdx.x; e < args.N; e += kThreads) S.bias[e] = args.bias[e];
    if (warp == 0) {   // two TMEM accumulators of BN fp32 columns x 128 lanes
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"((uint32_t)(2 * BN))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = S.tmem_base;
    constexpr uint32_t kTxBytes = (kBM + BN) * kBK * 2;

    // tile i of unit u: row block, column tile, split index and its K range
    auto tile_of = [&](int u, int i, int& m0, int& n0, int& z, int& kb, int& nkz) {
        int m, n;
        if (headed) { m = u; n = i; z = 0; }
        else {
            z = u / (mt * nt);
            const int r = u - z * mt * nt;
            m = r / nt;
            n = r - m * nt;
        }
        m0 = m * kBM;
        n0 = n * BN;
        kb = (int)(((long long)nk * z) / nsplit);
        nkz = (int)(((long long)nk * (z + 1)) / nsplit) - kb;
    };

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        int it = 0;
        bool ok = !args.withhold;
        for (int u = blockIdx.x; u < units && ok; u += gridDim.x)
            for (int i = 0; i < per_unit && ok; ++i) {
                int m0, n0, z, kb, nkz;
                tile_of(u, i, m0, n0, z, kb, nkz);
                for (int j = 0; j < nkz; ++j, ++it) {
                    const int s = it % kStages;
                    if (it >= kStages && !wait_or_abort(&S.empty[s], ((it / kStages) & 1) ^ 1, abort, args.err, lim)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&S.full[s], kTxBytes);
                    tma_load_2d(S.a[s], &map_a, (kb + j) * kBK, m0, &S.full[s]);
                    tma_load_2d(S.b[s], &map_b, (kb + j) * kBK, n0, &S.full[s]);
                }
            }
        S.issued = it;
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        constexpr uint32_t idesc = instr_desc(kBM, BN);
        int it = 0, lt = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < units && ok; u += gridDim.x)
            for (int i = 0; i < per_unit && ok; ++i, ++lt) {
                int m0, n0, z, kb, nkz;
                tile_of(u, i, m0, n0, z, kb, nkz);
                const int buf = lt & 1;
                if (lt >= 2 && !wait_or_abort(&S.acc_empty[buf], ((lt >> 1) & 1) ^ 1, abort, args.err, lim)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(buf * BN);
                for (int j = 0; j < nkz; ++j, ++it) {
                    const int s = it % kStages;
                    if (!wait_or_abort(&S.full[s], (it / kStages) & 1, abort, args.err, lim)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t ad = smem_desc(smem_u32(S.a[s])), bd = smem_desc(smem_u32(S.b[s]));
#pragma unroll
                    for (int k = 0; k < kBK / 16; ++k)    // advance 16 bf16 (32 B) along K inside the swizzle atom
                        umma_bf16(d, ad + 2 * k, bd + 2 * k, idesc, (j > 0 || k > 0) ? 1u : 0u);
                    umma_commit(&S.empty[s]);
                }
                if (ok) umma_commit(&S.acc_full[buf]);
            }
        umma_commit(&S.done);                  // arrives when every issued MMA has completed
    } else if (warp >= 2) {
        // ---------------- epilogue: TMEM -> bias + activation -> global (+ head)
        const int q = warp & 3, part = (warp - 2) >> 2;
        const int rl = q * 32 + lane;            // row of the tile = TMEM lane
        unsigned char* const stg = S.stage[warp - 2];
        int lt = 0, lu = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < units && ok; u += gridDim.x, ++lu) {
            float hs[kMaxHead] = {0.f, 0.f, 0.f, 0.f};
            for (int i = 0; i < per_unit && ok; ++i, ++lt) {
                int m0, n0, z, kb, nkz;
                tile_of(u, i, m0, n0, z, kb, nkz);
                const int buf = lt & 1;
                ok = __all_sync(0xFFFFFFFFu, wait_or_abort(&S.acc_full[buf], (lt >> 1) & 1, abort, args.err, lim));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                float* const out_f32 = args.ws ? args.ws + (size_t)z * args.M * args.ldc : args.out_f32;
                const int r0 = m0 + q * 32, r = r0 + lane;
                const bool live = r < args.M;
                const int rows_valid = min(32, args.M - r0);
                // staged (coalesced) stores when rows are 16-byte aligned; else one element at a time
                const int ldp = args.ldp ? args.ldp : args.ldc;
                const bool vf = args.ldc % 4 == 0 && (reinterpret_cast<uintptr_t>(out_f32) & 15) == 0;
                const bool vp = ldp % 4 == 0 && (reinterpret_cast<uintptr_t>(args.pre) & 15) == 0;
                const bool vb = args.ldc % 8 == 0 && (reinterpret_cast<uintptr_t>(args.out_bf16) & 15) == 0;
                const bool vt = args.ldt % 8 == 0 && (reinterpret_cast<uintptr_t>(args.out_bf16_t) & 15) == 0;
                // the layer's ELU values leave it only as bf16 (inference hidden layers, a head's input)
                const bool packed_elu = args.act == SF_ACT_ELU && !args.pre && !out_f32 && (args.out_bf16 || headed);
#pragma unroll 1
                for (int c = part; c < BN / 32; c += kParts) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + c * 32), v);
                    const int nb = n0 + c * 32;
                    if (nb >= args.N) continue;                    // uniform across the warp
                    const bool full = nb + 32 <= args.N;
                    if (args.bias) {
                        if (full && bias_smem) {
                            const float4* b4 = reinterpret_cast<const float4*>(S.bias + nb);
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const float4 b = b4[k];
                                v[4 * k] += b.x; v[4 * k + 1] += b.y; v[4 * k + 2] += b.z; v[4 * k + 3] += b.w;
                            }
                        } else if (full) {
                            const float4* b4 = reinterpret_cast<const float4*>(args.bias + nb);
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const float4 b = __ldg(b4 + k);
                                v[4 * k] += b.x; v[4 * k + 1] += b.y; v[4 * k + 2] += b.z; v[4 * k + 3] += b.w;
                            }
                        } else {
#pragma unroll
                            for (int k = 0; k < 32; ++k)
                                if (nb + k < args.N) v[k] += args.bias[nb + k];
                        }
                    }
                    const size_t row = (size_t)r * args.ldc + nb;
                    if (packed_elu) {   // ELU in packed bf16 when only bf16 values leave this layer
                        uint32_t pk[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) pk[e] = elu_bf16x2(__float_as_uint(v[2 * e]), __float_as_uint(v[2 * e + 1]));
                        if (args.out_bf16) {
                            if (full && vb) {
                                uint4 w[4];
#pragma unroll
                                for (int k = 0; k < 4; ++k) w[k] = make_uint4(pk[4 * k], pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
                                stage_store(stg, w, reinterpret_cast<unsigned char*>(args.out_bf16 + (size_t)r0 * args.ldc + nb),
                                            (size_t)args.ldc * 2, rows_valid, lane);
                            } else if (live) {
#pragma unroll
                                for (int k = 0; k < 32; ++k)
                                    if (nb + k < args.N)
                                        args.out_bf16[row + k] = __ushort_as_bfloat16((unsigned short)(pk[k >> 1] >> (16 * (k & 1))));
                            }
                        }
                        if (args.out_bf16_t) {   // the same bf16 values transposed (a training forward)
                            if (full && rows_valid == 32 && vt) {
                                __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(stg);
#pragma unroll
                                for (int h = 0; h < 2; ++h) {
#pragma unroll
                                    for (int kk = 0; kk < 16; ++kk) {
                                        const int k = 16 * h + kk;
                                        sb[kk * 32 + lane] = __ushort_as_bfloat16((unsigned short)(pk[k >> 1] >> (16 * (k & 1))));
                                    }
                                    __syncwarp();
#pragma unroll
                                    for (int i = 0; i < 2; ++i) {
                                        const int kk = (lane >> 2) + 8 * i, piece = lane & 3;
                                        const uint4 x = *reinterpret_cast<const uint4*>(stg + kk * 64 + piece * 16);
                                        *reinterpret_cast<uint4*>(args.out_bf16_t + (size_t)(nb + 16 * h + kk) * args.ldt +
                                                                  r0 + piece * 8) = x;
                                    }
                                    __syncwarp();
                                }
                            } else if (live) {
#pragma unroll
                                for (int k = 0; k < 32; ++k)
                                    if (nb + k < args.N)
                                        args.out_bf16_t[(size_t)(nb + k) * args.ldt + r] =
                                            __ushort_as_bfloat16((unsigned short)(pk[k >> 1] >> (16 * (k & 1))));
                            }
                        }
                        if (headed) {   // the same bf16 activations times the head weights, columns in order
                            const float* hw = &S.hw[0][nb];    // weights beyond N are zero
#pragma unroll
                            for (int k = 0; k < 32; k += 2) {
                                const float x0 = __uint_as_float(pk[k >> 1] << 16), x1 = __uint_as_float(pk[k >> 1] & 0xFFFF0000u);
#pragma unroll
                                for (int j = 0; j < kMaxHead; ++j)
                                    if (j < args.H) {
                                        const float2 w2 = *reinterpret_cast<const float2*>(hw + j * kHeadMaxN + k);
                                        hs[j] = fmaf(x1, w2.y, fmaf(x0, w2.x, hs[j]));
                                    }
                            }
                        }
                        continue;
                    }
                    if (args.pre) {
                        if (full && vp) {
                            stage_store_f32(stg, v, args.pre + (size_t)r0 * ldp + nb, ldp, rows_valid, lane);
                        } else if (live) {
                            const size_t prow = (size_t)r * ldp + nb;
#pragma unroll
                            for (int k = 0; k < 32; ++k)
                                if (nb + k < args.N) args.pre[prow + k] = v[k];
                        }
                    }
                    activate32(v, args.act);
                    if (out_f32) {
                        if (full && vf) {
                            stage_store_f32(stg, v, out_f32 + (size_t)r0 * args.ldc + nb, args.ldc, rows_valid, lane);
                        } else if (live) {
#pragma unroll
                            for (int k = 0; k < 32; ++k)
                                if (nb + k < args.N) out_f32[row + k] = v[k];
                        }
                    }
                    if (args.out_bf16) {
                        if (full && vb) {
                            stage_store_bf16(stg, v, args.out_bf16 + (size_t)r0 * args.ldc + nb, args.ldc, rows_valid,
                                             lane);
                        } else if (live) {
#pragma unroll
                            for (int k = 0; k < 32; ++k)
                                if (nb + k < args.N) args.out_bf16[row + k] = __float2bfloat16_rn(v[k]);
                        }
                    }
                    if (args.out_bf16_t && full && rows_valid == 32 && vt) {
                        // staged: 16 columns at a time through the warp's buffer (column k's 32 rows are
                        // 64 contiguous bytes of the transpose), then 16-byte stores
                        __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(stg);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
#pragma unroll
                            for (int kk = 0; kk < 16; ++kk) sb[kk * 32 + lane] = __float2bfloat16_rn(v[16 * h + kk]);
                            __syncwarp();
#pragma unroll
                            for (int i = 0; i < 2; ++i) {
                                const int kk = (lane >> 2) + 8 * i, piece = lane & 3;
                                const uint4 x = *reinterpret_cast<const uint4*>(stg + kk * 64 + piece * 16);
                                *reinterpret_cast<uint4*>(args.out_bf16_t + (size_t)(nb + 16 * h + kk) * args.ldt + r0 +
                                                          piece * 8) = x;
                            }
                            __syncwarp();
                        }
                    } else if (args.out_bf16_t && live) {   // lanes hold consecutive rows: each column store is contiguous
#pragma unroll
                        for (int k = 0; k < 32; ++k)
                            if (nb + k < args.N) args.out_bf16_t[(size_t)(nb + k) * args.ldt + r] = __float2bfloat16_rn(v[k]);
                    }
                    if (headed) {   // the bf16-rounded activations times the head weights, columns in order
                        const float* hw = &S.hw[0][nb];    // weights beyond N are zero
#pragma unroll
                        for (int k = 0; k < 32; k += 2) {
                            uint32_t p;
                            asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(p) : "f"(v[k + 1]), "f"(v[k]));
                            const float x0 = __uint_as_float(p << 16), x1 = __uint_as_float(p & 0xFFFF0000u);
#pragma unroll
                            for (int j = 0; j < kMaxHead; ++j)
                                if (j < args.H) {
                                    const float2 w2 = *reinterpret_cast<const float2*>(hw + j * kHeadMaxN + k);
                                    hs[j] = fmaf(x1, w2.y, fmaf(x0, w2.x, hs[j]));
                                }
                        }
                    }
                }
                const bool last = i == per_unit - 1;
                if (headed && last && part > 0) {   // hand the partials to part 0's thread of this row
                    const int p = lu & 1;
#pragma unroll
                    for (int j = 0; j < kMaxHead; ++j) S.head[p][part - 1][rl][j] = hs[j];
                    mbar_arrive(&S.head_full[p]);
                }
                if (headed && last && part == 0) {
                    const int p = lu & 1;
                    ok = __all_sync(0xFFFFFFFFu, wait_or_abort(&S.head_full[p], (lu >> 1) & 1, abort, args.err, lim));
                    if (ok && r < args.M) {
#pragma unroll
                        for (int j = 0; j < kMaxHead; ++j)
                            if (j < args.H) {
                                float sum = hs[j];   // parts in order
#pragma unroll
                                for (int k = 0; k < kParts - 1; ++k) sum += S.head[p][k][rl][j];
                                args.head_out[(size_t)r * args.ldh + j] =
                                    activate1(sum + (args.head_b ? args.head_b[j] : 0.f), args.head_act);
                            }
                    }
                }
                // release the accumulator (part 0 only after reading the head partials, so that the
                // other parts cannot overwrite them before: they must first receive a later tile)
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.acc_empty[buf]);
            }
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();   // every role has finished or given up: abort and issued are final
    // every issued MMA completes (done is committed on every path)
    mbar_wait(&S.done, 0, args.err, SF_GEMM_TIMEOUT);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN))
                     : "memory");
    }
    // after an abort, the TMA loads still in flight must land before exit
    // (bounded by the default 1 s, whatever limit the caller set)
    if (threadIdx.x == 0 && S.abort) {
        const int n = S.issued;
        for (int s = 0; s < kStages && s < n; ++s) {
            const int last = ((n - 1 - s) / kStages) * kStages + s;     // last K tile loaded into stage s
            mbar_wait(&S.full[s], (last / kStages) & 1, nullptr, 0);
        }
    }
}

// ---------------------------------------------------------------- host: tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// bf16 matrix [rows, cols] row-major (cols contiguous), box 64 x box_rows, 128-byte swizzle
bool make_map(CUtensorMap* m, const void* base, int rows, int cols, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// streaming multiprocessors of the current device (looked up once per device)
int sm_count() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        cached[dev] = n;
    }
    return cached[dev];
}

template <int BN>
cudaError_t launch_bn(const GemmArgs& g0, cudaStream_t s) {
    constexpr int ST = stages_for<BN>();
    CUtensorMap ma, mb;
    if (!make_map(&ma, g0.A, g0.M, g0.K, kBM) || !make_map(&mb, g0.B, g0.Nb, g0.K, BN)) return cudaErrorInvalidValue;
    GemmArgs g = g0;
    const int nk = (g.K + kBK - 1) / kBK;
    g.splits = g.ws ? std::max(1, std::min(g.splits, nk)) : 1;
    const long long mt = (g.M + kBM - 1) / kBM, nt = (g.N + BN - 1) / BN;
    const long long units = g.head_w ? mt : mt * nt * g.splits;
    const int grid = (int)std::min<long long>(units, sm_count());
    static_assert(sizeof(GemmSmem<BN, ST>) + 1024 <= 227 * 1024, "GEMM shared memory above the per-CTA limit");
    using Smem = GemmSmem<BN, ST>;
    static_assert(offsetof(Smem, stage) % 16 == 0 && offsetof(Smem, hw) % 16 == 0 && offsetof(Smem, bias) % 16 == 0,
                  "vector-accessed shared memory must be 16-byte aligned");
    const size_t smem = sizeof(GemmSmem<BN, ST>) + 1024;
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(tc_gemm_kernel<BN, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    tc_gemm_kernel<BN, ST><<<grid, kThreads, smem, s>>>(ma, mb, g);
    return cudaGetLastError();
}

}  // namespace

cudaError_t sf_gemm_launch(const GemmArgs& g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if (g.K <= 0 || g.K % 8 != 0 || g.Nb < 1) return cudaErrorInvalidValue;
    // split-K partial sums are plain products: no bias, activation or extra outputs
    if (g.ws && (g.bias || g.pre || g.out_bf16 || g.out_bf16_t || g.act != SF_ACT_NONE || g.splits < 1))
        return cudaErrorInvalidValue;
    // the fused head: inference only, at most four outputs
    if (g.head_w && (g.ws || !g.head_out || g.H < 1 || g.H > kMaxHead || g.ldh < g.H || g.ldhw < g.N ||
                     g.N > kHeadMaxN))
        return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(g.A) | reinterpret_cast<uintptr_t>(g.B)) & 15) return cudaErrorInvalidValue;
    switch (g.bn) {
        case 64: return launch_bn<64>(g, s);
        case 128: return launch_bn<128>(g, s);
        case 256: return launch_bn<256>(g, s);
        default: return cudaErrorInvalidValue;
    }
}
