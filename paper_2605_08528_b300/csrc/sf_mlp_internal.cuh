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
// the same on the input src's last training forward converted (same input width): m's layer 0
// reads src's bf16 copies, which must stay unchanged until m's backward has run
sf_status sf_mlp_forward_train_shared_on(sf_mlp_handle m, sf_mlp_handle src, cudaStream_t stream, int batch,
                                         float* d_y, int ldy);
// ends m's borrow of another network's input (after its backward)
void sf_mlp_end_share(sf_mlp_handle m);
// weight and bias gradients of the last training forward from the upstream gradient d_dy [batch][ldy]
sf_status sf_mlp_backward_on(sf_mlp_handle m, cudaStream_t stream, const float* d_dy, int ldy, int batch);
// adds the sum of squares of every gradient into *d_acc
sf_status sf_mlp_grad_sumsq_on(sf_mlp_handle m, cudaStream_t stream, float* d_acc);
// Adam (0.9, 0.999, 1e-8) with learning rate *d_lr and gradients scaled by *d_scale
sf_status sf_mlp_adam_on(sf_mlp_handle m, cudaStream_t stream, const float* d_lr, const float* d_scale);
int sf_mlp_out_dim(sf_mlp_handle m);
int sf_mlp_in_dim(sf_mlp_handle m);
