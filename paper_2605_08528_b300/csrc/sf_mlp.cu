// sf_mlp.cu -- BF16 MLPs on the tensor cores: inference and training (Adam).
//
// An MLP of L dense layers y = act_l(W_l x + b_l) keeps fp32 master weights,
// bf16 copies W_l [out, in] (forward) and W_l^T [in, out] (backward), and for
// a training batch the bf16 layer inputs X_l [B, in], their transposes X_l^T
// and the fp32 pre-activations Z_l [B, out].  Every product runs in the
// tcgen05 GEMM of sf_gemm.cu (C = act(A B^T + bias)):
//   forward   X_{l+1} = act(X_l W_l^T + b_l)          A = X_l,      B = W_l
//   weights   dW_l    = dZ_l^T X_l                     A = dZ_l^T,   B = X_l^T
//   inputs    dX_l    = dZ_l W_l                       A = dZ_l,     B = W_l^T
// with dZ_l = dX_{l+1} * act'(Z_l) computed elementwise, bias gradients by a
// column reduction, and an Adam step that refreshes both bf16 copies.  Widths
// are padded to multiples of 8 (the GEMM's 16-byte row rule) with zeros.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sf.h"
#include "sf_gemm.cuh"
#include "sf_mlp_internal.cuh"

namespace {

constexpr int kMaxLayers = 8;
constexpr int kSplitMax = 16;   // split-K partials of a weight gradient (K = the batch rows)

int pad8(int x) { return (x + 7) & ~7; }

__device__ __forceinline__ float act_grad(float z, int act) {
    switch (act) {
        case SF_ACT_ELU: return z > 0.f ? 1.f : expf(z);
        case SF_ACT_SILU: {
            const float s = 1.f / (1.f + expf(-z));
            return s * (1.f + z * (1.f - s));
        }
        case SF_ACT_TANH: {
            const float t = tanhf(z);
            return 1.f - t * t;
        }
        default: return 1.f;
    }
}
// the same from the layer's bf16 output h = act(z) where that determines it: ELU
// (1 for h > 0, else h + 1 = exp(z)), tanh (1 - h^2), identity
__device__ __forceinline__ float act_grad_out(float h, int act) {
    switch (act) {
        case SF_ACT_ELU: return h > 0.f ? 1.f : h + 1.f;
        case SF_ACT_TANH: return 1.f - h * h;
        default: return 1.f;
    }
}


// x [B, n] f32 -> bf16 [B, ld] with n == ld, ld % 8 == 0 and 16-byte rows: 8 elements per thread
__global__ void to_bf16_vec8_kernel(const float* __restrict__ x, size_t n8, __nv_bfloat16* __restrict__ y) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n8) return;
    const float4 a = reinterpret_cast<const float4*>(x)[2 * i], b = reinterpret_cast<const float4*>(x)[2 * i + 1];
    __nv_bfloat162 h[4] = {__floats2bfloat162_rn(a.x, a.y), __floats2bfloat162_rn(a.z, a.w),
                           __floats2bfloat162_rn(b.x, b.y), __floats2bfloat162_rn(b.z, b.w)};
    reinterpret_cast<uint4*>(y)[i] = *reinterpret_cast<const uint4*>(h);
}

// x [B, n] f32 -> bf16 [B, ld] (zero padded) and optionally bf16^T [ld, B]
// x [B, n] f32 (row stride ldx) -> bf16 y [B, ld] (zero padded) and, when yt is set, y^T [ld, B]:
// 32 x 32 tiles through shared memory so that both the rows and the transpose are written
// coalesced (block 32 x 8, grid (ld / 32, B / 32) rounded up)
__global__ void to_bf16_kernel(const float* __restrict__ x, int B, int n, int ldx, __nv_bfloat16* __restrict__ y,
                               int ld, __nv_bfloat16* __restrict__ yt) {
    __shared__ __nv_bfloat16 tile[32][34];
    const int c0 = blockIdx.x * 32, b0 = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int b = b0 + ty + 8 * j, c = c0 + tx;
        __nv_bfloat16 v = __float2bfloat16_rn(0.f);
        if (b < B && c < ld) {
            v = __float2bfloat16_rn(c < n ? x[(size_t)b * ldx + c] : 0.f);
            y[(size_t)b * ld + c] = v;
        }
        tile[ty + 8 * j][tx] = v;
    }
    if (!yt) return;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = c0 + ty + 8 * j, b = b0 + tx;
        if (b < B && c < ld) yt[(size_t)c * B + b] = tile[tx][ty + 8 * j];
    }
}
// dZ = dA * act'(Z) (dA fp32, or bf16 dAb for a hidden layer; Z null: act' from the bf16
// output H [B, ld]) as bf16 [B, ld] and its transpose dZ^T [ld, B] (32 x 32 tiles
// through shared memory), and the partial column sums of the bf16 dZ for the bias
// gradient: block (x, s) covers columns [32 x, 32 x + 32) of rows [kBackRows s,
// kBackRows (s + 1)); thread (ty, tx) adds its rows of column tx in order, then the
// 8 row threads are added in order: part[s][c] (c < n)
constexpr int kBackRows = 128;
__global__ void act_back_kernel(const float* __restrict__ dA, const __nv_bfloat16* __restrict__ dAb,
                                const float* __restrict__ Z,
                                const __nv_bfloat16* __restrict__ H, int B, int n, int ld, int act,
                                __nv_bfloat16* __restrict__ dz, __nv_bfloat16* __restrict__ dzt,
                                float* __restrict__ part) {
    __shared__ __nv_bfloat16 tile[32][34];
    __shared__ float red[8][33];
    const int c0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;
    const int rb = blockIdx.y * kBackRows;
    float acc = 0.f;
    for (int b0 = rb; b0 < rb + kBackRows && b0 < B; b0 += 32) {   // block-uniform
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = b0 + ty + 8 * j, c = c0 + tx;
            __nv_bfloat16 v = __float2bfloat16_rn(0.f);
            if (b < B && c < ld) {
                float g = 0.f;
                if (c < n) {
                    const size_t i = (size_t)b * ld + c;
                    const float up = dAb ? __bfloat162float(dAb[i]) : dA[i];
                    g = up * (Z ? act_grad(Z[i], act) : act_grad_out(__bfloat162float(H[i]), act));
                }
                v = __float2bfloat16_rn(g);
                dz[(size_t)b * ld + c] = v;
            }
            acc += __bfloat162float(v);
            tile[ty + 8 * j][tx] = v;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + ty + 8 * j, b = b0 + tx;
            if (b < B && c < ld) dzt[(size_t)c * B + b] = tile[tx][ty + 8 * j];
        }
        __syncthreads();   // the tile is rewritten by the next 32 rows
    }
    red[ty][tx] = acc;
    __syncthreads();
    if (ty == 0) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += red[k][tx];
        const int c = c0 + tx;
        if (c < n) part[(size_t)blockIdx.y * n + c] = t;
    }
}

// mean-squared-error gradient of the output: dY = 2 (y - t) / (B n)
__global__ void mse_grad_kernel(const float* __restrict__ y, const float* __restrict__ t, int B, int n, int ld,
                                int ldt, float* __restrict__ dy) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (size_t)B * ld) {
        const int b = (int)(i / ld), c = (int)(i % ld);
        const float d = c < n ? y[i] - t[(size_t)b * ldt + c] : 0.f;
        dy[i] = 2.f * d / ((float)B * (float)n);
    }
}

// the loss mean (y - t)^2 over the B x n outputs, in a fixed order: thread k
// sums elements k, k + 256, ... and the 256 sums meet in a tree (one block;
// launched only for the step whose loss is read)
__global__ void mse_loss_kernel(const float* __restrict__ y, const float* __restrict__ t, int B, int n, int ld,
                                int ldt, float* __restrict__ loss) {
    __shared__ float red[256];
    float l = 0.f;
    for (size_t i = threadIdx.x; i < (size_t)B * n; i += 256) {
        const int b = (int)(i / n), c = (int)(i % n);
        const float d = y[(size_t)b * ld + c] - t[(size_t)b * ldt + c];
        l += d * d;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / ((float)B * (float)n);
}

// the bias gradient: db[c] = the S partial column sums of act_back_kernel, one warp per
// column: lane l adds partials l, l + 32, ... in order, then the lanes meet in a fixed
// butterfly, so the sum is the same on every run
__global__ void bias_sum_kernel(const float* __restrict__ part, int n, int S, float* __restrict__ db) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= n) return;   // warp-uniform
    float t = 0.f;
    for (int s = lane; s < S; s += 32) t += part[(size_t)s * n + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    if (lane == 0) db[c] = t;
}

// Adam (Kingma & Ba) on fp32 masters; refresh bf16 W [out, ldi] and W^T [ldi, ldo]
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2,
                            int out, int in, int ldi, int ldo, __nv_bfloat16* __restrict__ wb,
                            __nv_bfloat16* __restrict__ wbt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) {   // weight matrix element (o, k) of [out, in]
        const int o = i / in, k = i % in;
        const __nv_bfloat16 hb = __float2bfloat16_rn(wi);
        wb[(size_t)o * ldi + k] = hb;
        wbt[(size_t)k * ldo + o] = hb;
    }
}

// sum of the split-K partials [S][out][ldi] into the dense [out, in] weight gradient (fixed order)
__global__ void reduce_compact_kernel(const float* __restrict__ ws, int S, int out, int in, int ldi,
                                      float* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= out * in) return;
    const size_t src = (size_t)(i / in) * ldi + (i % in), stride = (size_t)out * ldi;
    float acc = 0.f;
    for (int z = 0; z < S; ++z) acc += ws[z * stride + src];
    dst[i] = acc;
}

// gather the fp32 weight gradient [out, ldi] into the dense [out, in] layout
__global__ void compact_kernel(const float* __restrict__ src, int out, int in, int ldi, float* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= out * in) return;
    dst[i] = src[(size_t)(i / in) * ldi + (i % in)];
}

__global__ void weights_to_bf16_kernel(const float* __restrict__ w, int out, int in, int ldi, int ldo,
                                       __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wbt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= out * in) return;
    const int o = i / in, k = i % in;
    const __nv_bfloat16 hb = __float2bfloat16_rn(w[i]);
    wb[(size_t)o * ldi + k] = hb;
    wbt[(size_t)k * ldo + o] = hb;
}

unsigned grid1(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }
// launch shape of the tiled [B, ld] kernels (to_bf16_kernel, act_back_kernel)
dim3 tgrid(int B, int ld) { return dim3((unsigned)((ld + 31) / 32), (unsigned)((B + 31) / 32)); }
const dim3 kTBlock(32, 8);

}  // namespace

struct sf_mlp {
    int L = 0;
    int dim[kMaxLayers + 1] = {};   // true widths
    int ld[kMaxLayers + 1] = {};    // padded widths
    int hidden_act = 0, out_act = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<void*> allocs;
    // parameters
    float* w[kMaxLayers] = {};      // fp32 [out, in]
    float* b[kMaxLayers] = {};      // fp32 [out]
    __nv_bfloat16* wb[kMaxLayers] = {};    // [out, ld_in], zero padded
    __nv_bfloat16* wbt[kMaxLayers] = {};   // [ld_in, ld_out]
    float *gw[kMaxLayers] = {}, *gb[kMaxLayers] = {};
    float *mw[kMaxLayers] = {}, *vw[kMaxLayers] = {}, *mb[kMaxLayers] = {}, *vb[kMaxLayers] = {};
    int adam_t = 0;
    // batch buffers
    int cap = 0;
    __nv_bfloat16* x[kMaxLayers + 1] = {};   // [cap, ld_l]
    __nv_bfloat16* xt[kMaxLayers + 1] = {};  // [ld_l, cap]
    float* z[kMaxLayers] = {};               // [cap, ld_{l+1}]
    float* y = nullptr;                      // [cap, ld_L] output f32
    float* dA = nullptr;                     // [cap, max ld] f32: the output layer's upstream gradient
    __nv_bfloat16* dAb = nullptr;            // [cap, max ld] bf16: a hidden layer's (the dX product of the layer above)
    __nv_bfloat16 *dz = nullptr, *dzt = nullptr;
    float* gwfull = nullptr;                 // [max out, max ld] f32 (padded gradient)
    float* ws = nullptr;                     // [kSplitMax][max out][max ld] f32 split-K partials of dW
    float* bpart = nullptr;                  // [cap / kBackRows][max ld] f32 partial bias gradients
    float* loss = nullptr;
    float* red = nullptr;                    // [kSumsqBlocks] partial sums of the gradient norm
    const sf_mlp* share = nullptr;           // while set: layer 0 reads its bf16 input (and its transpose) from it
    unsigned* errw = nullptr;
    unsigned long long wait_ns = 0;          // GEMM ring-wait limit (0: 1 s)
    int withhold = 0;                        // GEMMs issue no operand loads (timeout test)
};

namespace {

sf_status mfail(sf_mlp* m, sf_status s, const std::string& e) {
    if (m) m->err = e;
    return s;
}

template <class T>
cudaError_t malloc_zero(sf_mlp* m, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
    if (e != cudaSuccess) return e;
    m->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return cudaMemset(q, 0, count * sizeof(T) + 16);
}

int act_of(const sf_mlp* m, int l) { return l == m->L - 1 ? m->out_act : m->hidden_act; }
// the training forward keeps layer l's fp32 pre-activation for the backward only where the
// derivative needs it: the output layer and SiLU (ELU, tanh and the identity follow from the
// bf16 output the next layer reads)
bool keeps_pre(const sf_mlp* m, int l) { return l == m->L - 1 || act_of(m, l) == SF_ACT_SILU; }

int tile_for(int n) { return n >= 256 ? 256 : (n > 64 ? 128 : 64); }

cudaError_t gemm(sf_mlp* m, const __nv_bfloat16* A, const __nv_bfloat16* B, const float* bias, int M, int N, int Nb,
                 int K, int act, float* pre, float* out_f32, __nv_bfloat16* out_bf16, __nv_bfloat16* out_t, int ldc,
                 int ldt, cudaStream_t st = nullptr, bool use_st = false, int ldp = 0) {
    GemmArgs g{};
    g.ldp = ldp;
    g.A = A; g.B = B; g.bias = bias; g.pre = pre; g.out_f32 = out_f32; g.out_bf16 = out_bf16; g.out_bf16_t = out_t;
    g.M = M; g.N = N; g.Nb = Nb; g.K = K; g.ldc = ldc; g.ldt = ldt; g.act = act; g.bn = tile_for(N); g.err = m->errw;
    g.wait_ns = m->wait_ns; g.withhold = m->withhold;
    return sf_gemm_launch(g, use_st ? st : m->stream);
}

// inference with a narrow last layer (at most 4 outputs): that layer runs in the
// epilogue of the layer before it (the GEMM's fused head), which then stores no
// activations: C_head = out_act(bf16(act(X W^T + b)) . W_last^T + b_last)
bool head_fusable(const sf_mlp* m) { return m->L >= 2 && m->dim[m->L] <= 4; }

// layer L - 2 with layer L - 1 as its fused head, into y [B][ldy]
cudaError_t gemm_head(sf_mlp* m, const __nv_bfloat16* A, int B, float* y, int ldy, cudaStream_t st) {
    const int l = m->L - 2;
    GemmArgs g{};
    g.A = A; g.B = m->wb[l]; g.bias = m->b[l];
    g.M = B; g.N = m->dim[l + 1]; g.Nb = m->dim[l + 1]; g.K = m->ld[l]; g.ldc = m->ld[l + 1]; g.act = m->hidden_act;
    g.bn = tile_for(g.N); g.err = m->errw; g.wait_ns = m->wait_ns; g.withhold = m->withhold;
    g.head_w = m->wb[l + 1]; g.ldhw = m->ld[l + 1]; g.head_b = m->b[l + 1]; g.head_out = y; g.ldh = ldy;
    g.H = m->dim[m->L]; g.head_act = m->out_act;
    return sf_gemm_launch(g, st);
}

cudaError_t ensure_batch(sf_mlp* m, int B) {
    if (B <= m->cap) return cudaSuccess;
    // buffers of a smaller batch stay allocated until destroy; the new set replaces them
    int maxld = 0;
    for (int l = 0; l <= m->L; ++l) maxld = maxld > m->ld[l] ? maxld : m->ld[l];
    cudaError_t e = cudaSuccess;
    for (int l = 0; l <= m->L && e == cudaSuccess; ++l) {
        e = malloc_zero(m, &m->x[l], (size_t)B * m->ld[l]);
        if (e == cudaSuccess) e = malloc_zero(m, &m->xt[l], (size_t)B * m->ld[l]);
    }
    for (int l = 0; l < m->L && e == cudaSuccess; ++l) e = malloc_zero(m, &m->z[l], (size_t)B * m->ld[l + 1]);
    if (e == cudaSuccess) e = malloc_zero(m, &m->y, (size_t)B * m->ld[m->L]);
    if (e == cudaSuccess) e = malloc_zero(m, &m->dA, (size_t)B * maxld);
    if (e == cudaSuccess) e = malloc_zero(m, &m->dAb, (size_t)B * maxld);
    if (e == cudaSuccess) e = malloc_zero(m, &m->dz, (size_t)B * maxld);
    if (e == cudaSuccess) e = malloc_zero(m, &m->dzt, (size_t)B * maxld);
    if (e == cudaSuccess) e = malloc_zero(m, &m->bpart, (size_t)((B + kBackRows - 1) / kBackRows) * maxld);
    if (e == cudaSuccess) m->cap = B;
    return e;
}

// the bf16 input of layer l and its transpose (layer 0 may borrow another network's)
const __nv_bfloat16* x_in(const sf_mlp* m, int l) { return l == 0 && m->share ? m->share->x[0] : m->x[l]; }
const __nv_bfloat16* xt_in(const sf_mlp* m, int l) { return l == 0 && m->share ? m->share->xt[0] : m->xt[l]; }

// forward of a batch already converted into x[0] (and xt[0] when training); the
// last layer writes y_out [B][ldy] (m->y with its padded width when null)
cudaError_t forward_core(sf_mlp* m, int B, bool train, float* y_out = nullptr, int ldy = 0,
                         cudaStream_t st = nullptr, bool use_st = false) {
    cudaError_t e = cudaSuccess;
    const bool fuse = !train && head_fusable(m);
    for (int l = 0; l < m->L && e == cudaSuccess; ++l) {
        const bool last = l == m->L - 1;
        if (fuse && l == m->L - 2) {
            e = gemm_head(m, x_in(m, l), B, y_out ? y_out : m->y, y_out ? ldy : m->ld[m->L], use_st ? st : m->stream);
            break;
        }
        // the pre-activations keep the layer's own row stride whatever the output's (the backward reads them
        // so); a hidden layer whose activation's derivative follows from its bf16 output keeps none
        e = gemm(m, x_in(m, l), m->wb[l], m->b[l], B, m->dim[l + 1], m->dim[l + 1], m->ld[l], act_of(m, l),
                 train && keeps_pre(m, l) ? m->z[l] : nullptr, last ? (y_out ? y_out : m->y) : nullptr, last ? nullptr : m->x[l + 1],
                 (train && !last) ? m->xt[l + 1] : nullptr, (last && y_out) ? ldy : m->ld[l + 1], B, st, use_st,
                 m->ld[l + 1]);
    }
    return e;
}

// upstream gradient dy [B, n] (row stride ldy) -> dA [B, ld] with zero padding
__global__ void dy_in_kernel(const float* __restrict__ dy, int B, int n, int ldy, int ld, float* __restrict__ dA) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)B * ld) return;
    const int b = (int)(i / ld), c = (int)(i % ld);
    dA[i] = c < n ? dy[(size_t)b * ldy + c] : 0.f;
}

// dW_l = dZ_l^T X_l [out, in] with K = B rows: the output has few tiles, so the K range is split over
// up to kSplitMax CTAs per tile (enough to fill the GPU) and the partials summed in a fixed order
cudaError_t weight_grad(sf_mlp* m, int l, int B, const __nv_bfloat16* dzt, cudaStream_t st) {
    const int o = m->dim[l + 1], li = m->ld[l], i = m->dim[l];
    const int bn = tile_for(li);
    const int tiles = ((o + 127) / 128) * ((li + bn - 1) / bn), nk = (B + 63) / 64;
    const int S = std::max(1, std::min(std::min(kSplitMax, nk), 296 / std::max(1, tiles)));
    GemmArgs g{};
    g.A = dzt; g.B = xt_in(m, l); g.M = o; g.N = li; g.Nb = li; g.K = B; g.ldc = li; g.act = SF_ACT_NONE;
    g.bn = bn; g.err = m->errw; g.wait_ns = m->wait_ns; g.withhold = m->withhold;
    if (S > 1) { g.ws = m->ws; g.splits = S; } else { g.out_f32 = m->gwfull; }
    cudaError_t e = sf_gemm_launch(g, st);
    if (e != cudaSuccess) return e;
    if (S > 1)
        reduce_compact_kernel<<<(unsigned)(((size_t)o * i + 255) / 256), 256, 0, st>>>(m->ws, S, o, i, li, m->gw[l]);
    else
        compact_kernel<<<(unsigned)(((size_t)o * i + 255) / 256), 256, 0, st>>>(m->gwfull, o, i, li, m->gw[l]);
    return cudaGetLastError();
}

// backward of the activations kept by the last training forward, from dA (holding dL/dy);
// with dx0 set, also the gradient with respect to the input, dX_0 = dZ_0 W_0, as
// fp32 [B][lddx] (ld[0] columns, the padding ones zero)
cudaError_t backward_core(sf_mlp* m, int B, cudaStream_t st, float* dx0 = nullptr, int lddx = 0) {
    cudaError_t e = cudaSuccess;
    for (int l = m->L - 1; l >= 0 && e == cudaSuccess; --l) {
        const int o = m->dim[l + 1], lo = m->ld[l + 1], li = m->ld[l];
        const int S = (B + kBackRows - 1) / kBackRows;   // partial bias sums, one per kBackRows rows
        act_back_kernel<<<dim3((unsigned)((lo + 31) / 32), (unsigned)S), kTBlock, 0, st>>>(
            m->dA, l == m->L - 1 ? nullptr : m->dAb, keeps_pre(m, l) ? m->z[l] : nullptr, m->x[l + 1], B, o, lo,
            act_of(m, l), m->dz, m->dzt, m->bpart);
        bias_sum_kernel<<<(unsigned)((o + 7) / 8), 256, 0, st>>>(m->bpart, o, S, m->gb[l]);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = weight_grad(m, l, B, m->dzt, st);
        if (e == cudaSuccess && l > 0)
            e = gemm(m, m->dz, m->wbt[l], nullptr, B, li, li, lo, SF_ACT_NONE, nullptr, nullptr, m->dAb, nullptr, li,
                     0, st, true);
        else if (e == cudaSuccess && dx0)
            e = gemm(m, m->dz, m->wbt[0], nullptr, B, li, li, lo, SF_ACT_NONE, nullptr, dx0, nullptr, nullptr, lddx,
                     0, st, true);
    }
    return e;
}

// every parameter tensor of a network as one index space: segment k holds
// n = off[k + 1] - off[k] values; weight segments also carry their bf16 copies
constexpr int kSegMax = 2 * kMaxLayers;
struct Segs {
    float* w[kSegMax];
    const float* g[kSegMax];
    float* m[kSegMax];
    float* v[kSegMax];
    __nv_bfloat16* wb[kSegMax];    // null for a bias
    __nv_bfloat16* wbt[kSegMax];
    int in[kSegMax], ldi[kSegMax], ldo[kSegMax];
    long long off[kSegMax + 1];
    int nseg;
};
__device__ __forceinline__ int seg_of(const Segs& S, long long i) {
    int k = 0;
    while (k + 1 < S.nseg && S.off[k + 1] <= i) ++k;
    return k;
}

// sum of squares of the gradients, deterministic: block j sums its fixed chunk
// of the index space (each thread a fixed stride, the warps added in order)
// into part[j]; sumsq_final adds the parts in order into *acc
constexpr int kSumsqBlocks = 148;
__global__ void sumsq_part_kernel(const Segs S, float* __restrict__ part) {
    __shared__ float red[8];
    const long long total = S.off[S.nseg];
    const long long chunk = (total + gridDim.x - 1) / gridDim.x;
    const long long i0 = (long long)blockIdx.x * chunk, i1 = min(total, i0 + chunk);
    float acc = 0.f;
    long long i = i0 + threadIdx.x;
    int k = i < i1 ? seg_of(S, i) : 0;
    for (; i < i1; i += blockDim.x) {
        while (S.off[k + 1] <= i) ++k;
        const float gi = S.g[k][i - S.off[k]];
        acc += gi * gi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}
__global__ void sumsq_final_kernel(const float* __restrict__ part, int P, float* __restrict__ acc) {
    if (threadIdx.x != 0) return;
    float t = 0.f;
    for (int j = 0; j < P; ++j) t += part[j];
    *acc += t;
}

// Adam (Kingma & Ba) over every tensor of a network in one launch, with the
// learning rate and a gradient scale read from device memory; weight elements
// (o, k) of [out, in] refresh their bf16 copies W [out, ldi] and W^T [ldi, ldo]
__global__ void adam_all_kernel(const Segs S, const float* __restrict__ lr_p, const float* __restrict__ scale_p,
                                float b1, float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.off[S.nseg]) return;
    const int k = seg_of(S, i);
    const long long j = i - S.off[k];
    const float gi = S.g[k][j] * *scale_p;
    const float mi = b1 * S.m[k][j] + (1.f - b1) * gi;
    const float vi = b2 * S.v[k][j] + (1.f - b2) * gi * gi;
    S.m[k][j] = mi;
    S.v[k][j] = vi;
    const float wi = S.w[k][j] - *lr_p * (mi / c1) / (sqrtf(vi / c2) + eps);
    S.w[k][j] = wi;
    if (S.wb[k]) {
        const int o = (int)(j / S.in[k]), c = (int)(j % S.in[k]);
        const __nv_bfloat16 hb = __float2bfloat16_rn(wi);
        S.wb[k][(size_t)o * S.ldi[k] + c] = hb;
        S.wbt[k][(size_t)c * S.ldo[k] + o] = hb;
    }
}

// the segment table of network m: per layer its weights, then its biases
Segs segs_of(const sf_mlp* m) {
    Segs S{};
    long long off = 0;
    int k = 0;
    for (int l = 0; l < m->L; ++l) {
        const int o = m->dim[l + 1], i = m->dim[l];
        S.w[k] = m->w[l]; S.g[k] = m->gw[l]; S.m[k] = m->mw[l]; S.v[k] = m->vw[l];
        S.wb[k] = m->wb[l]; S.wbt[k] = m->wbt[l]; S.in[k] = i; S.ldi[k] = m->ld[l]; S.ldo[k] = m->ld[l + 1];
        S.off[k] = off; off += (long long)o * i; ++k;
        S.w[k] = m->b[l]; S.g[k] = m->gb[l]; S.m[k] = m->mb[l]; S.v[k] = m->vb[l];
        S.wb[k] = nullptr; S.wbt[k] = nullptr; S.in[k] = 1; S.ldi[k] = 0; S.ldo[k] = 0;
        S.off[k] = off; off += o; ++k;
    }
    S.off[k] = off;
    S.nseg = k;
    return S;
}

}  // namespace

// ---------------------------------------------------------------- static scratch
// Scratch of sf_mlp_forward_static: a fixed device array in this library's
// image (every GPU that loads the library holds it until the process exits).
constexpr size_t kStaticScratchBytes = (size_t)4 << 20;
static __device__ __align__(256) unsigned char g_mlp_static_scratch[kStaticScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// device address of the static scratch on the current device, looked up once per device
cudaError_t static_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_mlp_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// bytes of static scratch one forward of `batch` rows needs
size_t static_need(const sf_mlp* m, int batch) {
    size_t n = 0;
    for (int l = 0; l < m->L; ++l) n += round256((size_t)batch * m->ld[l] * 2);
    return n + round256((size_t)batch * m->ld[m->L] * 4);
}

}  // namespace

extern "C" {

sf_status sf_mlp_forward_static(sf_mlp_handle m, const float* d_x, int ldx, int batch, float* d_y, int ldy) {
    if (!m || !d_x || !d_y || batch < 0 || ldx < m->dim[0] || ldy < m->dim[m->L]) return SF_ERR_INVALID_ARG;
    // the address lookup comes first, so that a call with batch 0 primes the
    // device (before any stream capture) without touching any buffer
    void* base = nullptr;
    cudaError_t e = static_scratch(&base);
    if (e != cudaSuccess) return mfail(m, SF_ERR_CUDA, std::string("static scratch: ") + cudaGetErrorString(e));
    if (batch == 0) return SF_OK;
    const size_t need = static_need(m, batch);
    if (need > kStaticScratchBytes)
        return mfail(m, SF_ERR_INVALID_ARG,
                     "sf_mlp_forward_static: batch " + std::to_string(batch) + " needs " + std::to_string(need) +
                         " bytes of scratch; the static scratch holds " + std::to_string(kStaticScratchBytes));
    // carve: bf16 input of every layer, then the fp32 output; zero it (padding columns must read as 0)
    unsigned char* p = static_cast<unsigned char*>(base);
    __nv_bfloat16* xs[kMaxLayers] = {};
    for (int l = 0; l < m->L; ++l) {
        xs[l] = reinterpret_cast<__nv_bfloat16*>(p);
        p += round256((size_t)batch * m->ld[l] * 2);
    }
    float* y = reinterpret_cast<float*>(p);
    e = cudaMemsetAsync(base, 0, need, m->stream);
    if (e == cudaSuccess) {
        to_bf16_kernel<<<tgrid(batch, m->ld[0]), kTBlock, 0, m->stream>>>(d_x, batch, m->dim[0], ldx, xs[0],
                                                                               m->ld[0], nullptr);
        e = cudaGetLastError();
    }
    for (int l = 0; l < m->L && e == cudaSuccess; ++l) {
        const bool last = l == m->L - 1;
        if (head_fusable(m) && l == m->L - 2) {   // the same layer sequence as sf_mlp_forward
            e = gemm_head(m, xs[l], batch, y, m->ld[m->L], m->stream);
            break;
        }
        e = gemm(m, xs[l], m->wb[l], m->b[l], batch, m->dim[l + 1], m->dim[l + 1], m->ld[l], act_of(m, l), nullptr,
                 last ? y : nullptr, last ? nullptr : xs[l + 1], nullptr, m->ld[l + 1], batch);
    }
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(d_y, (size_t)ldy * 4, y, (size_t)m->ld[m->L] * 4, (size_t)m->dim[m->L] * 4, batch,
                              cudaMemcpyDeviceToDevice, m->stream);
    return e == cudaSuccess ? SF_OK
                            : mfail(m, SF_ERR_CUDA, std::string("sf_mlp_forward_static: ") + cudaGetErrorString(e));
}

size_t sf_mlp_static_scratch_bytes(void) { return kStaticScratchBytes; }

sf_status sf_mlp_create(int num_layers, const int32_t* dims, int hidden_act, int out_act, void* cuda_stream,
                        sf_mlp_handle* out) {
    if (!out || !dims || num_layers < 1 || num_layers > kMaxLayers) return SF_ERR_INVALID_ARG;
    *out = nullptr;
    for (int l = 0; l <= num_layers; ++l)
        if (dims[l] < 1 || dims[l] > 4096) return SF_ERR_INVALID_ARG;
    if (hidden_act < 0 || hidden_act > 3 || out_act < 0 || out_act > 3) return SF_ERR_INVALID_ARG;
    sf_mlp* m = new sf_mlp();
    m->L = num_layers;
    for (int l = 0; l <= num_layers; ++l) { m->dim[l] = dims[l]; m->ld[l] = pad8(dims[l]); }
    m->hidden_act = hidden_act;
    m->out_act = out_act;
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = malloc_zero(m, &m->errw, 1);
    if (e == cudaSuccess) e = malloc_zero(m, &m->loss, 1);
    if (e == cudaSuccess) e = malloc_zero(m, &m->red, 256);
    int maxo = 0, maxi = 0;
    for (int l = 0; l < num_layers && e == cudaSuccess; ++l) {
        const int o = dims[l + 1], i = dims[l];
        maxo = maxo > m->ld[l + 1] ? maxo : m->ld[l + 1];
        maxi = maxi > m->ld[l] ? maxi : m->ld[l];
        e = malloc_zero(m, &m->w[l], (size_t)o * i);
        if (e == cudaSuccess) e = malloc_zero(m, &m->b[l], (size_t)o);
        if (e == cudaSuccess) e = malloc_zero(m, &m->wb[l], (size_t)o * m->ld[l]);
        if (e == cudaSuccess) e = malloc_zero(m, &m->wbt[l], (size_t)m->ld[l] * m->ld[l + 1]);
        if (e == cudaSuccess) e = malloc_zero(m, &m->gw[l], (size_t)o * i);
        if (e == cudaSuccess) e = malloc_zero(m, &m->gb[l], (size_t)o);
        if (e == cudaSuccess) e = malloc_zero(m, &m->mw[l], (size_t)o * i);
        if (e == cudaSuccess) e = malloc_zero(m, &m->vw[l], (size_t)o * i);
        if (e == cudaSuccess) e = malloc_zero(m, &m->mb[l], (size_t)o);
        if (e == cudaSuccess) e = malloc_zero(m, &m->vb[l], (size_t)o);
    }
    if (e == cudaSuccess) e = malloc_zero(m, &m->gwfull, (size_t)maxo * maxi);
    if (e == cudaSuccess) e = malloc_zero(m, &m->ws, (size_t)kSplitMax * maxo * maxi);
    if (e != cudaSuccess) {
        for (void* p : m->allocs) cudaFree(p);
        delete m;
        return e == cudaErrorMemoryAllocation ? SF_ERR_OOM : SF_ERR_CUDA;
    }
    *out = m;
    return SF_OK;
}

sf_status sf_mlp_destroy(sf_mlp_handle m) {
    if (!m) return SF_OK;
    cudaStreamSynchronize(m->stream);
    for (void* p : m->allocs) cudaFree(p);
    delete m;
    return SF_OK;
}

const char* sf_mlp_last_error(sf_mlp_handle m) { return m ? m->err.c_str() : ""; }

sf_status sf_mlp_set_layer(sf_mlp_handle m, int layer, const float* h_w, const float* h_b) {
    if (!m || layer < 0 || layer >= m->L || !h_w || !h_b) return SF_ERR_INVALID_ARG;
    const int o = m->dim[layer + 1], i = m->dim[layer];
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e == cudaSuccess) e = cudaMemcpy(m->w[layer], h_w, (size_t)o * i * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->b[layer], h_b, (size_t)o * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        weights_to_bf16_kernel<<<grid1((size_t)o * i), 256, 0, m->stream>>>(m->w[layer], o, i, m->ld[layer],
                                                                            m->ld[layer + 1], m->wb[layer],
                                                                            m->wbt[layer]);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? SF_OK : mfail(m, SF_ERR_CUDA, cudaGetErrorString(e));
}

sf_status sf_mlp_get_layer(sf_mlp_handle m, int layer, float* h_w, float* h_b, float* h_gw, float* h_gb) {
    if (!m || layer < 0 || layer >= m->L) return SF_ERR_INVALID_ARG;
    const int o = m->dim[layer + 1], i = m->dim[layer];
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e == cudaSuccess && h_w) e = cudaMemcpy(h_w, m->w[layer], (size_t)o * i * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_b) e = cudaMemcpy(h_b, m->b[layer], (size_t)o * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_gw) e = cudaMemcpy(h_gw, m->gw[layer], (size_t)o * i * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_gb) e = cudaMemcpy(h_gb, m->gb[layer], (size_t)o * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SF_OK : mfail(m, SF_ERR_CUDA, cudaGetErrorString(e));
}

sf_status sf_mlp_forward(sf_mlp_handle m, const float* d_x, int ldx, int batch, float* d_y, int ldy) {
    if (!m) return SF_ERR_INVALID_ARG;
    return sf_mlp_forward_on(m, m->stream, d_x, ldx, batch, d_y, ldy);
}

}  // extern "C"

sf_status sf_mlp_reserve(sf_mlp_handle m, int batch) {
    if (!m || batch < 0) return SF_ERR_INVALID_ARG;
    cudaError_t e = ensure_batch(m, batch);
    return e == cudaSuccess ? SF_OK : mfail(m, SF_ERR_OOM, "batch buffers");
}

sf_status sf_mlp_forward_on(sf_mlp_handle m, cudaStream_t stream, const float* d_x, int ldx, int batch, float* d_y,
                            int ldy) {
    if (!m || !d_x || !d_y || batch < 0 || ldx < m->dim[0] || ldy < m->dim[m->L]) return SF_ERR_INVALID_ARG;
    if (batch == 0) return SF_OK;
    cudaError_t e = ensure_batch(m, batch);
    if (e != cudaSuccess) return mfail(m, e == cudaErrorMemoryAllocation ? SF_ERR_OOM : SF_ERR_CUDA, "batch buffers");
    cudaStream_t saved = m->stream;
    m->stream = stream;
    m->share = nullptr;   // the network's own input from here on
    if (m->dim[0] == m->ld[0] && ldx == m->dim[0] && (reinterpret_cast<uintptr_t>(d_x) & 15) == 0) {
        const size_t n8 = (size_t)batch * m->ld[0] / 8;
        to_bf16_vec8_kernel<<<grid1(n8), 256, 0, stream>>>(d_x, n8, m->x[0]);
    } else {
        to_bf16_kernel<<<tgrid(batch, m->ld[0]), kTBlock, 0, stream>>>(d_x, batch, m->dim[0], ldx, m->x[0],
                                                                            m->ld[0], nullptr);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = forward_core(m, batch, false, d_y, ldy);
    m->stream = saved;
    return e == cudaSuccess ? SF_OK : mfail(m, SF_ERR_CUDA, std::string("sf_mlp_forward: ") + cudaGetErrorString(e));
}

extern "C" {

sf_status sf_mlp_train_step(sf_mlp_handle m, const float* d_x, const float* d_t, int batch, float lr, int update,
                            float* h_loss) {
    if (!m || !d_x || !d_t || batch < 8 || batch % 8 != 0) return SF_ERR_INVALID_ARG;
    cudaError_t e = ensure_batch(m, batch);
    if (e != cudaSuccess) return mfail(m, SF_ERR_OOM, "batch buffers");
    const int L = m->L, B = batch;
    m->share = nullptr;
    to_bf16_kernel<<<tgrid(B, m->ld[0]), kTBlock, 0, m->stream>>>(d_x, B, m->dim[0], m->dim[0], m->x[0], m->ld[0],
                                                                       m->xt[0]);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = forward_core(m, B, true);
    if (e == cudaSuccess) {
        mse_grad_kernel<<<grid1((size_t)B * m->ld[L]), 256, 0, m->stream>>>(m->y, d_t, B, m->dim[L], m->ld[L],
                                                                            m->dim[L], m->dA);
        if (h_loss)
            mse_loss_kernel<<<1, 256, 0, m->stream>>>(m->y, d_t, B, m->dim[L], m->ld[L], m->dim[L], m->loss);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = backward_core(m, B, m->stream);
    if (e == cudaSuccess && update) {
        ++m->adam_t;
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
        for (int l = 0; l < L && e == cudaSuccess; ++l) {
            const int o = m->dim[l + 1], i = m->dim[l];
            adam_kernel<<<grid1((size_t)o * i), 256, 0, m->stream>>>(m->w[l], m->gw[l], m->mw[l], m->vw[l], o * i, lr,
                                                                     b1, b2, eps, c1, c2, o, i, m->ld[l],
                                                                     m->ld[l + 1], m->wb[l], m->wbt[l]);
            adam_kernel<<<grid1(o), 256, 0, m->stream>>>(m->b[l], m->gb[l], m->mb[l], m->vb[l], o, lr, b1, b2, eps, c1,
                                                         c2, 0, 1, 0, 0, nullptr, nullptr);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && h_loss) {
        e = cudaMemcpyAsync(h_loss, m->loss, 4, cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    }
    return e == cudaSuccess ? SF_OK : mfail(m, SF_ERR_CUDA, std::string("sf_mlp_train_step: ") + cudaGetErrorString(e));
}

}  // extern "C"

sf_status sf_mlp_convert_train_on(sf_mlp_handle m, cudaStream_t st, const float* d_x, int ldx, int batch) {
    if (!m || !d_x || batch < 8 || batch % 8 != 0 || ldx < m->dim[0]) return SF_ERR_INVALID_ARG;
    cudaError_t e = ensure_batch(m, batch);
    if (e != cudaSuccess) return mfail(m, SF_ERR_OOM, "batch buffers");
    m->share = nullptr;
    to_bf16_kernel<<<tgrid(batch, m->ld[0]), kTBlock, 0, st>>>(d_x, batch, m->dim[0], ldx, m->x[0], m->ld[0],
                                                                    m->xt[0]);
    e = cudaGetLastError();
    return e == cudaSuccess ? SF_OK : mfail(m, SF_ERR_CUDA, std::string("forward_train: ") + cudaGetErrorString(e));
}

sf_status sf_mlp_forward_converted_on(sf_mlp_handle m, cudaStream_t st, int batch, float* d_y, int ldy) {
    if (!m || !d_y || batch < 8 || batch % 8 != 0 || batch > m->cap || ldy < m->dim[m->L]) return SF_ERR_INVALID_ARG;
    const cudaError_t e = forward_core(m, batch, true, d_y, ldy, st, true);
    return e == cudaSuccess ? SF_OK : mfail(m, SF_ERR_CUDA, std::string("forward_train: ") + cudaGetErrorString(e));
}

sf_status sf_mlp_forward_train_on(sf_mlp_handle m, cudaStream_t st, const float* d_x, int ldx, int batch, float* d_y,
                                  int ldy) {
    if (!m || !d_x || !d_y || batch < 8 || batch % 8 != 0 || ldx < m->dim[0] || ldy < m->dim[m->L])
        return SF_ERR_INVALID_ARG;
    const sf_status s = sf_mlp_convert_train_on(m, st, d_x, ldx, batch);
    return s == SF_OK ? sf_mlp_forward_converted_on(m, st, batch, d_y, ldy) : s;
}

void sf_mlp_end_share(sf_mlp_handle m) {
    if (m) m->share = nullptr;
}

sf_status sf_mlp_forward_train_shared_on(sf_mlp_handle m, sf_mlp_handle src, cudaStream_t st, int batch, float* d_y,
                                         int ldy) {
    if (!m || !src || m == src || !d_y || batch < 8 || batch % 8 != 0 || batch > src->cap ||
        m->dim[0] != src->dim[0] || ldy < m->dim[m->L])
        return SF_ERR_INVALID_ARG;
    cudaError_t e = ensure_batch(m, batch);
    if (e != cudaSuccess) return mfail(m, SF_ERR_OOM, "batch buffers");
    m->share = src;   // until the next forward_train of m with its own input
    e = forward_core(m, batch, true, d_y, ldy, st, true);
    return e == cudaSuccess ? SF_OK : mfail(m, SF_ERR_CUDA, std::string("forward_train: ") + cudaGetErrorString(e));
}

sf_status sf_mlp_backward_on(sf_mlp_handle m, cudaStream_t st, const float* d_dy, int ldy, int batch) {
    if (!m || !d_dy || batch < 8 || batch > m->cap || ldy < m->dim[m->L]) return SF_ERR_INVALID_ARG;
    const int L = m->L;
    dy_in_kernel<<<grid1((size_t)batch * m->ld[L]), 256, 0, st>>>(d_dy, batch, m->dim[L], ldy, m->ld[L], m->dA);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = backward_core(m, batch, st);
    return e == cudaSuccess ? SF_OK : mfail(m, SF_ERR_CUDA, std::string("backward: ") + cudaGetErrorString(e));
}

sf_status sf_mlp_backward_dx_on(sf_mlp_handle m, cudaStream_t st, const float* d_dy, int ldy, int batch, float* d_dx,
                                int lddx) {
    if (!m || !d_dy || !d_dx || batch < 8 || batch > m->cap || ldy < m->dim[m->L] || lddx < m->ld[0])
        return SF_ERR_INVALID_ARG;
    const int L = m->L;
    dy_in_kernel<<<grid1((size_t)batch * m->ld[L]), 256, 0, st>>>(d_dy, batch, m->dim[L], ldy, m->ld[L], m->dA);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = backward_core(m, batch, st, d_dx, lddx);
    return e == cudaSuccess ? SF_OK : mfail(m, SF_ERR_CUDA, std::string("backward: ") + cudaGetErrorString(e));
}

sf_status sf_mlp_grad_sumsq_on(sf_mlp_handle m, cudaStream_t st, float* d_acc) {
    if (!m || !d_acc) return SF_ERR_INVALID_ARG;
    sumsq_part_kernel<<<kSumsqBlocks, 256, 0, st>>>(segs_of(m), m->red);
    sumsq_final_kernel<<<1, 32, 0, st>>>(m->red, kSumsqBlocks, d_acc);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SF_OK : mfail(m, SF_ERR_CUDA, cudaGetErrorString(e));
}

sf_status sf_mlp_adam_on(sf_mlp_handle m, cudaStream_t st, const float* d_lr, const float* d_scale) {
    if (!m || !d_lr || !d_scale) return SF_ERR_INVALID_ARG;
    ++m->adam_t;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
    const Segs S = segs_of(m);
    adam_all_kernel<<<grid1((size_t)S.off[S.nseg]), 256, 0, st>>>(S, d_lr, d_scale, b1, b2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SF_OK : mfail(m, SF_ERR_CUDA, cudaGetErrorString(e));
}

sf_status sf_mlp_device_layer(sf_mlp_handle m, int layer, const void** d_wb, int* ld_in, const float** d_b) {
    if (!m || layer < 0 || layer >= m->L || !d_wb || !ld_in || !d_b) return SF_ERR_INVALID_ARG;
    *d_wb = m->wb[layer];
    *ld_in = m->ld[layer];
    *d_b = m->b[layer];
    return SF_OK;
}

int sf_mlp_out_dim(sf_mlp_handle m) { return m ? m->dim[m->L] : 0; }
int sf_mlp_in_dim(sf_mlp_handle m) { return m ? m->dim[0] : 0; }

extern "C" {

sf_status sf_mlp_sync(sf_mlp_handle m) {
    if (!m) return SF_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return mfail(m, SF_ERR_CUDA, cudaGetErrorString(e));
    unsigned w = 0;
    e = cudaMemcpy(&w, m->errw, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return mfail(m, SF_ERR_CUDA, cudaGetErrorString(e));
    if (w & SF_GEMM_TIMEOUT) {
        cudaMemset(m->errw, 0, 4);
        return mfail(m, SF_ERR_TIMEOUT, "a tensor-core GEMM gave up waiting for its operands");
    }
    return SF_OK;
}

sf_status sf_mlp_set_wait_limit(sf_mlp_handle m, unsigned long long limit_ns, int withhold_producer) {
    if (!m) return SF_ERR_INVALID_ARG;
    m->wait_ns = limit_ns == 0 ? 1ull : limit_ns;   // the kernels read 0 as the 1 s default
    m->withhold = withhold_producer != 0;
    return SF_OK;
}

sf_status sf_gemm_bf16(const void* d_a, const void* d_b, const float* d_bias, int M, int N, int K, int act,
                       float* d_out_f32, void* d_out_bf16, void* d_out_bf16_t, int ldc, int ldt, int tile_n,
                       unsigned* d_err, void* cuda_stream) {
    if (!d_a || !d_b || M < 0 || N < 0 || K <= 0 || K % 8 != 0 || act < 0 || act > 3) return SF_ERR_INVALID_ARG;
    if (tile_n != 64 && tile_n != 128 && tile_n != 256) return SF_ERR_INVALID_ARG;
    if (ldc < N && (d_out_f32 || d_out_bf16)) return SF_ERR_INVALID_ARG;
    if (ldt < M && d_out_bf16_t) return SF_ERR_INVALID_ARG;
    GemmArgs g{};
    g.A = static_cast<const __nv_bfloat16*>(d_a);
    g.B = static_cast<const __nv_bfloat16*>(d_b);
    g.bias = d_bias;
    g.out_f32 = d_out_f32;
    g.out_bf16 = static_cast<__nv_bfloat16*>(d_out_bf16);
    g.out_bf16_t = static_cast<__nv_bfloat16*>(d_out_bf16_t);
    g.M = M; g.N = N; g.Nb = N; g.K = K; g.ldc = ldc; g.ldt = ldt; g.act = act; g.bn = tile_n; g.err = d_err;
    cudaError_t e = sf_gemm_launch(g, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? SF_OK : (e == cudaErrorInvalidValue ? SF_ERR_INVALID_ARG : SF_ERR_CUDA);
}

}  // extern "C"
