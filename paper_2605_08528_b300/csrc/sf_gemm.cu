// sf_gemm.cu -- BF16 tensor-core GEMM with a fused epilogue for the MLPs (sm_103a).
//
//   C[M, N] = act(A[M, K] . B[N, K]^T + bias[N])
//
// A and B are bf16, row-major with K contiguous (B is a weight matrix stored
// [out, in]); accumulation is fp32.  One CTA computes a 128 x BN tile:
//   warp 0 lane 0  issues TMA loads of 128 x 64 (A) and BN x 64 (B) K-tiles
//                  into a STAGES-deep ring (128-byte swizzle);
//   warp 1 lane 0  issues tcgen05.mma (M 128, N BN, K 16) into a TMEM
//                  accumulator of BN fp32 columns and commits each stage back;
//   warps 0-7      read the accumulator with tcgen05.ld (warp w owns rows
//                  32(w%4)..32(w%4)+31 and every other 32-column chunk), add
//                  the bias, apply the activation and store.
// Every mbarrier wait is bounded: on expiry the kernel records SF_GEMM_TIMEOUT
// in the error word and stops issuing work; before it frees its TMEM and
// returns it waits (bounded, 1 s) for every MMA it issued and for every TMA
// load it issued, so no asynchronous copy outlives the CTA.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "sf_gemm.cuh"
#include "sf_tc.cuh"

namespace {

constexpr int kBM = 128, kBK = 64, kThreads = 256;   // 8 warps: 2 per TMEM lane slice
// Pipeline depth: a deep ring (4 stages, one CTA per SM) for long K; for short K
// (few K tiles per CTA) a shallow ring that lets two CTAs share an SM (shared
// memory and TMEM columns), so one CTA's epilogue overlaps the other's main loop
constexpr int kDeep = 4;
template <int BN>
constexpr int shallow_for() { return BN >= 256 ? 2 : (BN >= 128 ? 3 : 4); }
constexpr int kShallowMaxK = 8;   // K tiles per CTA up to which the shallow ring is used
using namespace sftc;

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned* err,
                                          uint64_t limit_ns = kWaitNs) {
    return sftc::mbar_wait(bar, parity, err, SF_GEMM_TIMEOUT, limit_ns);
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

template <int BN, int kStages>
struct alignas(1024) GemmSmem {
    __nv_bfloat16 a[kStages][kBM * kBK];
    __nv_bfloat16 b[kStages][BN * kBK];
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t done;
    uint32_t tmem_base;
    uint32_t abort;    // a ring wait gave up (producer or MMA issuer)
    int issued;        // K tiles whose TMA loads the producer issued
};

template <int BN, int kStages>
__global__ void __launch_bounds__(kThreads, kStages == kDeep ? 1 : 2)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                   const GemmArgs args) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    GemmSmem<BN, kStages>& S = *reinterpret_cast<GemmSmem<BN, kStages>*>(
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int nk = (args.K + kBK - 1) / kBK;
    // split K: CTA z of gridDim.z takes K tiles [kb, kb + nkz) and writes its partial sum to the workspace
    const int z = blockIdx.z, nsplit = gridDim.z;
    const int kb = (int)(((long long)nk * z) / nsplit), nkz = (int)(((long long)nk * (z + 1)) / nsplit) - kb;
    float* const out_f32 = args.ws ? args.ws + (size_t)z * args.M * args.ldc : args.out_f32;

    const uint64_t lim = args.wait_ns ? args.wait_ns : kWaitNs;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) { mbar_init(&S.full[s], 1); mbar_init(&S.empty[s], 1); }
        mbar_init(&S.done, 1);
        S.abort = 0;
        S.issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {   // TMEM accumulator: BN fp32 columns x 128 lanes
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = S.tmem_base;
    constexpr uint32_t kTxBytes = (kBM + BN) * kBK * 2;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        int j = 0;
        for (; j < nkz && !args.withhold; ++j) {
            const int s = j % kStages, kt = kb + j;
            if (j >= kStages && !mbar_wait(&S.empty[s], ((j / kStages) & 1) ^ 1, args.err, lim)) {
                S.abort = 1;
                break;
            }
            mbar_expect_tx(&S.full[s], kTxBytes);
            tma_load_2d(S.a[s], &map_a, kt * kBK, m0, &S.full[s]);
            tma_load_2d(S.b[s], &map_b, kt * kBK, n0, &S.full[s]);
        }
        S.issued = j;
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        constexpr uint32_t idesc = instr_desc(kBM, BN);
        bool ok = true;
        for (int j = 0; j < nkz && ok; ++j) {
            const int s = j % kStages;
            ok = mbar_wait(&S.full[s], (j / kStages) & 1, args.err, lim);
            if (!ok) {
                S.abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t ad = smem_desc(smem_u32(S.a[s])), bd = smem_desc(smem_u32(S.b[s]));
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)    // advance 16 bf16 (32 B) along K inside the swizzle atom
                umma_bf16(tmem, ad + 2 * k, bd + 2 * k, idesc, (j > 0 || k > 0) ? 1u : 0u);
            umma_commit(&S.empty[s]);
        }
        umma_commit(&S.done);                  // arrives when every issued MMA has completed
    }
    __syncwarp();
    __syncthreads();   // the producer and the MMA issuer are done: abort and issued are final

    // ---------------- epilogue: TMEM -> bias + activation -> global
    // every issued MMA completes (done is committed on every path), then the
    // accumulator is used only if no wait gave up
    const bool fin = __all_sync(0xFFFFFFFFu, mbar_wait(&S.done, 0, args.err));
    const bool have = fin && S.abort == 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int r = m0 + (warp & 3) * 32 + lane;   // TMEM lane slice of this warp
    // 16-byte vector stores when rows are aligned for them
    const bool vf = args.ldc % 4 == 0 && ((reinterpret_cast<uintptr_t>(out_f32) |
                                          reinterpret_cast<uintptr_t>(args.pre)) & 15) == 0;
    const bool vb = args.ldc % 8 == 0 && (reinterpret_cast<uintptr_t>(args.out_bf16) & 15) == 0;
    if (have) {
#pragma unroll 1
        for (int c = warp >> 2; c < BN / 32; c += kThreads / 128) {   // the two warp halves split the columns
            float v[32];
            tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(c * 32), v);
            const int nb = n0 + c * 32;
            if (r >= args.M || nb >= args.N) continue;
            const bool full = nb + 32 <= args.N;
            if (args.bias) {
                if (full) {
                    const float4* b4 = reinterpret_cast<const float4*>(args.bias + nb);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 b = __ldg(b4 + q);
                        v[4 * q] += b.x; v[4 * q + 1] += b.y; v[4 * q + 2] += b.z; v[4 * q + 3] += b.w;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (nb + i < args.N) v[i] += args.bias[nb + i];
                }
            }
            const size_t row = (size_t)r * args.ldc + nb;
            if (args.pre) {
                if (full && vf) {
                    float4* p4 = reinterpret_cast<float4*>(args.pre + row);
#pragma unroll
                    for (int q = 0; q < 8; ++q) p4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (nb + i < args.N) args.pre[row + i] = v[i];
                }
            }
            activate32(v, args.act);
            if (out_f32) {
                if (full && vf) {
                    float4* p4 = reinterpret_cast<float4*>(out_f32 + row);
#pragma unroll
                    for (int q = 0; q < 8; ++q) p4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (nb + i < args.N) out_f32[row + i] = v[i];
                }
            }
            if (args.out_bf16) {
                if (full && vb) {
                    uint4* p4 = reinterpret_cast<uint4*>(args.out_bf16 + row);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint32_t w[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * q + 2 * k], v[8 * q + 2 * k + 1]);
                            w[k] = *reinterpret_cast<const uint32_t*>(&h2);
                        }
                        p4[q] = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (nb + i < args.N) args.out_bf16[row + i] = __float2bfloat16_rn(v[i]);
                }
            }
            if (args.out_bf16_t) {   // lanes hold consecutive rows: each column store is contiguous across the warp
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (nb + i < args.N) args.out_bf16_t[(size_t)(nb + i) * args.ldt + r] = __float2bfloat16_rn(v[i]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
    }
    // after a timeout, the TMA loads still in flight must land before exit
    // (bounded by the default 1 s, whatever limit the caller set)
    if (threadIdx.x == 0 && !have) {
        const int n = S.issued;
        for (int s = 0; s < kStages && s < n; ++s) {
            const int last = ((n - 1 - s) / kStages) * kStages + s;     // last K tile loaded into stage s
            mbar_wait(&S.full[s], (last / kStages) & 1, nullptr);
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

template <int BN, int ST>
cudaError_t launch_st(const CUtensorMap& ma, const CUtensorMap& mb, const GemmArgs& g, dim3 grid, cudaStream_t s) {
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

template <int BN>
cudaError_t launch_bn(const GemmArgs& g, cudaStream_t s) {
    CUtensorMap ma, mb;
    if (!make_map(&ma, g.A, g.M, g.K, kBM) || !make_map(&mb, g.B, g.Nb, g.K, BN)) return cudaErrorInvalidValue;
    const int nk = (g.K + kBK - 1) / kBK;
    const int splits = g.ws ? std::max(1, std::min(g.splits, nk)) : 1;
    dim3 grid((g.N + BN - 1) / BN, (g.M + kBM - 1) / kBM, splits);
    if ((nk + splits - 1) / splits <= kShallowMaxK) return launch_st<BN, shallow_for<BN>()>(ma, mb, g, grid, s);
    return launch_st<BN, kDeep>(ma, mb, g, grid, s);
}

}  // namespace

cudaError_t sf_gemm_launch(const GemmArgs& g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if (g.K <= 0 || g.K % 8 != 0 || g.Nb < 1) return cudaErrorInvalidValue;
    // split-K partial sums are plain products: no bias, activation or extra outputs
    if (g.ws && (g.bias || g.pre || g.out_bf16 || g.out_bf16_t || g.act != SF_ACT_NONE || g.splits < 1))
        return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(g.A) | reinterpret_cast<uintptr_t>(g.B)) & 15) return cudaErrorInvalidValue;
    switch (g.bn) {
        case 64: return launch_bn<64>(g, s);
        case 128: return launch_bn<128>(g, s);
        case 256: return launch_bn<256>(g, s);
        default: return cudaErrorInvalidValue;
    }
}
