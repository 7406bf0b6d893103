// sf_mlp_internal.cuh -- MLP calls on an explicit stream (used by the step graph).
#pragma once
#include <cuda_runtime.h>

#include "../../include/sf.h"

// make sure the batch buffers of `batch` rows exist (allocates; not capturable)
sf_status sf_mlp_reserve(sf_mlp_handle m, int batch);
// sf_mlp_forward on `stream` instead of the MLP's own stream (no allocation if reserved)
sf_status sf_mlp_forward_on(sf_mlp_handle m, cudaStream_t stream, const float* d_x, int ldx, int batch, float* d_y,
                            int ldy);

// the late-fusion actor-critic on an explicit stream (used by the policy step and its graph)
sf_status sf_lf_reserve(sf_lf_handle m, int batch);
sf_status sf_lf_forward_on(sf_lf_handle m, cudaStream_t stream, const float* d_obs, const int32_t* d_n_road,
                           const int32_t* d_n_veh, int num_agents, float* d_mean, float* d_value, float* d_embed);

// training pieces on an explicit stream (used by the PPO engine)
// forward of `batch` rows keeping the activations the backward needs; outputs d_y [batch][ldy]
sf_status sf_mlp_forward_train_on(sf_mlp_handle m, cudaStream_t stream, const float* d_x, int ldx, int batch,
                                  float* d_y, int ldy);
// the same in two parts: the input converted into m's bf16 copies (and their transpose), then
// the forward on them (another network may read the converted input meanwhile, as below)
sf_status sf_mlp_convert_train_on(sf_mlp_handle m, cudaStream_t stream, const float* d_x, int ldx, int batch);
sf_status sf_mlp_forward_converted_on(sf_mlp_handle m, cudaStream_t stream, int batch, float* d_y, int ldy);
// the same on the input src's last training forward converted (same input width): m's layer 0
// reads src's bf16 copies, which must stay unchanged until m's backward has run
sf_status sf_mlp_forward_train_shared_on(sf_mlp_handle m, sf_mlp_handle src, cudaStream_t stream, int batch,
                                         float* d_y, int ldy);
// ends m's borrow of another network's input (after its backward)
void sf_mlp_end_share(sf_mlp_handle m);
// weight and bias gradients of the last training forward from the upstream gradient d_dy [batch][ldy]
sf_status sf_mlp_backward_on(sf_mlp_handle m, cudaStream_t stream, const float* d_dy, int ldy, int batch);
// the same, and the gradient with respect to the input of the last training forward,
// d_dx [batch][lddx] fp32 (lddx >= the input width padded to 8; padding columns zero)
sf_status sf_mlp_backward_dx_on(sf_mlp_handle m, cudaStream_t stream, const float* d_dy, int ldy, int batch,
                                float* d_dx, int lddx);
// adds the sum of squares of every gradient into *d_acc
sf_status sf_mlp_grad_sumsq_on(sf_mlp_handle m, cudaStream_t stream, float* d_acc);
// Adam (0.9, 0.999, 1e-8) with learning rate *d_lr and gradients scaled by *d_scale
sf_status sf_mlp_adam_on(sf_mlp_handle m, cudaStream_t stream, const float* d_lr, const float* d_scale);
// device copies of layer `layer`: bf16 weights [out][*ld_in] (zero padded) and fp32 bias [out]
sf_status sf_mlp_device_layer(sf_mlp_handle m, int layer, const void** d_wb, int* ld_in, const float** d_b);
int sf_mlp_out_dim(sf_mlp_handle m);
int sf_mlp_in_dim(sf_mlp_handle m);

// Training of the late-fusion actor-critic (sf_lf.cu): the ego encoders and
// trunks (with their heads) as MLPs, the set encoders' masters with the
// arg-max backward; it keeps the sf_lf handle's inference weights up to date.
struct LfTrainer;
sf_status lft_create(sf_lf_handle lf, cudaStream_t stream, LfTrainer** out);
void lft_destroy(LfTrainer* t);
const char* lft_error(LfTrainer* t);
// forward of `rows` rows (obs [rows][1929], group counts) keeping what the backward needs:
// d_mean [rows][3], d_value [rows]
sf_status lft_forward(LfTrainer* t, const float* d_obs, const int32_t* d_n_road, const int32_t* d_n_veh, int rows,
                      float* d_mean, float* d_value);
// every parameter's gradient from d_dmean [rows][3] and d_dvalue [rows] (after lft_forward)
sf_status lft_backward(LfTrainer* t, const float* d_dmean, const float* d_dvalue, int rows);
sf_status lft_grad_sumsq(LfTrainer* t, float* d_acc);
// Adam on every parameter (learning rate *d_lr, gradients scaled by *d_scale); the set
// encoders' inference images follow at once, the dense layers at lft_publish
sf_status lft_adam(LfTrainer* t, const float* d_lr, const float* d_scale);
sf_status lft_publish(LfTrainer* t);
// the last forward's maximising slots into d_out [2 groups][2 networks][rows][96] (0xFFFF: empty group)
sf_status lft_argmax(LfTrainer* t, uint16_t* d_out);
// parameters / last gradients in the sf_lf flat layout without the 3 log-stds (synchronous)
sf_status lft_get(LfTrainer* t, float* h_params, float* h_grads);
