// sf_gemm.cuh -- arguments of the BF16 tensor-core GEMM (sf_gemm.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/sf.h"   // SF_ACT_* activation codes
#define SF_GEMM_TIMEOUT 2u   // error-word bit: a bounded mbarrier wait gave up

// C[M, N] = act(A[M, K] . B[N, K]^T + bias[N]); A, B bf16 row-major, K % 8 == 0,
// 16-byte aligned bases.  Rows of A beyond M and of B beyond Nb read as zero.
struct GemmArgs {
    const __nv_bfloat16* A;   // [M, K]
    const __nv_bfloat16* B;   // [Nb, K]
    const float* bias;        // [N] or null
    float* pre;               // [M, ldc] pre-activation (f32) or null
    float* out_f32;           // [M, ldc] or null
    __nv_bfloat16* out_bf16;  // [M, ldc] or null
    __nv_bfloat16* out_bf16_t;// [N, ldt] transposed or null
    int M, N, Nb, K;
    int ldc, ldt;
    int ldp;                  // row stride of pre (0: ldc)
    int act;
    int bn;                   // tile width 64, 128 or 256
    unsigned* err;            // device error word (SF_GEMM_TIMEOUT)
    // split K (optional): with ws set, `splits` CTAs share each output tile's K range and
    // split z writes its partial product to ws + z * M * ldc (no bias, activation or other
    // outputs); the caller sums the partials.  splits is capped at the number of K tiles.
    int splits;
    float* ws;
    // bounded waits: the operand-ring waits give up after wait_ns of wall time
    // (0: 1 s); withhold != 0 issues no TMA load at all, so the first wait runs
    // out on a barrier nothing completes (a test of the timeout path)
    unsigned long long wait_ns;
    int withhold;
    // fused narrow head (optional; no split K): with head_w set, every row's
    // activated values, rounded to bf16, are also multiplied by the bf16 head
    // weights head_w [H][ldhw] (columns 0..N-1 used) and summed over all N
    // columns; the CTA that owns a row block computes all of its column tiles,
    // so each row's sum is formed in one fixed order (column tiles in order,
    // each thread's columns in order, then the two column halves of a tile) and
    //   head_out[r * ldh + j] = head_act(sum_j + head_b[j]),  j < H <= 4.
    // The layer's own outputs (out_f32, out_bf16, ...) may be null.
    const __nv_bfloat16* head_w;
    const float* head_b;
    float* head_out;
    int H, ldhw, ldh, head_act;
};

cudaError_t sf_gemm_launch(const GemmArgs& g, cudaStream_t s);
