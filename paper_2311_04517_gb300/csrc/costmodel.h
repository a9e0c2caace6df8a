// Launchers of the cost-model kernels (costmodel.cu), internal.
#pragma once

#include <stddef.h>

#include "kernels.h"

// ---- cost model of the objective's search forms (costmodel.cu) ----
// Floats of per-block gradient scratch for N samples.
size_t hpc_cm_part_floats(int N);
// Loss and gradient (m == nullptr: written to grad_out / loss_out), or one
// Adam step on params / m / v with bias corrections bc1 = 1 - beta1^t,
// bc2 = 1 - beta2^t (loss_out, nullable, gets the loss before the step).
int hpc_cm_grad_launch(const hpc_launch &L, const float *params, const float *feats,
                       const float *targets, int N, float *part, float *m, float *v, float lr,
                       float bc1, float bc2, float *grad_out, float *loss_out);
int hpc_cm_predict_launch(const hpc_launch &L, const float *params, const float *feats, int N,
                          float *out);
