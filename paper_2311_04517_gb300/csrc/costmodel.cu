// Cost model of the objective's search forms: a two-hidden-layer ReLU
// perceptron that predicts ln(ns per row) of a form from the inputs the host
// builds (dims, cluster count, padding, centroid separation, form), trained
// on measured times with full-batch Adam.  Everything the network computes
// runs in the kernels below: the forward pass, back-propagation of the mean
// squared error, the reduction of the per-sample gradients and the Adam
// update (Kingma and Ba 2015: first and second moments, bias corrections
// 1 - beta^t, step lr * m_hat / (sqrt(v_hat) + eps)).
//
// The network is tiny (1377 parameters) and its data a few hundred
// measurements, so the kernels aim at determinism, not speed: one thread per
// sample, per-block gradient sums taken in sample order in shared memory,
// then one thread per parameter adding the block sums in block order.  Two
// launches per training step.
//
// Flat parameter layout: W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.
#include "../../include/hpclust.h"
#include "costmodel.h"

namespace {

constexpr int F = HPC_CM_NFEAT;
constexpr int H = HPC_CM_HIDDEN;
constexpr int P = HPC_CM_NPARAM;
constexpr int OW1 = 0, OB1 = H * F, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H,
              OB3 = OW3 + H;
static_assert(OB3 + 1 == P, "parameter layout");
constexpr int CB = 64;  // samples (threads) per block of the gradient kernel
constexpr int HS = H + 1;  // padded row stride of the per-sample activations

// Forward pass of one sample with the parameters in shared memory; fills
// h1, h2 (post-ReLU) and returns y.
__device__ __forceinline__ float cm_forward(const float *sp, const float *x, float *h1,
                                            float *h2) {
  for (int j = 0; j < H; ++j) {
    float z = 0.0f;
    for (int f = 0; f < F; ++f) z = fmaf(sp[OW1 + j * F + f], x[f], z);
    z += sp[OB1 + j];
    h1[j] = fmaxf(z, 0.0f);
  }
  for (int j = 0; j < H; ++j) {
    float z = 0.0f;
    for (int i = 0; i < H; ++i) z = fmaf(sp[OW2 + j * H + i], h1[i], z);
    z += sp[OB2 + j];
    h2[j] = fmaxf(z, 0.0f);
  }
  float y = 0.0f;
  for (int j = 0; j < H; ++j) y = fmaf(sp[OW3 + j], h2[j], y);
  return y + sp[OB3];
}

// Per-block sums of the per-sample gradients of (y - t)^2 (the 1/N of the
// mean comes in the reduction) and of the squared residuals:
// part[blk * (P + 1) + p], p = P holding the residual sum.
__global__ void __launch_bounds__(CB) cm_grad_kernel(const float *__restrict__ params,
                                                     const float *__restrict__ feats,
                                                     const float *__restrict__ targets, int N,
                                                     float *__restrict__ part) {
  __shared__ float sp[P];
  __shared__ float sx[CB][F];
  __shared__ float sh1[CB][HS], sh2[CB][HS], sd1[CB][HS], sd2[CB][HS];
  __shared__ float sgy[CB], sr2[CB];
  const int tid = threadIdx.x;
  for (int p = tid; p < P; p += CB) sp[p] = params[p];
  const int64_t n = (int64_t)blockIdx.x * CB + tid;
  const bool valid = n < N;
  for (int f = 0; f < F; ++f) sx[tid][f] = valid ? feats[n * F + f] : 0.0f;
  __syncthreads();

  const float y = cm_forward(sp, sx[tid], sh1[tid], sh2[tid]);
  const float r = valid ? y - targets[n] : 0.0f;
  const float gy = 2.0f * r;  // d(r^2)/dy
  sgy[tid] = gy;
  sr2[tid] = r * r;
  // output layer -> second hidden layer (ReLU passes where its output is > 0)
  for (int j = 0; j < H; ++j) sd2[tid][j] = sh2[tid][j] > 0.0f ? gy * sp[OW3 + j] : 0.0f;
  // second -> first hidden layer: delta1 = (W2^T delta2) masked
  for (int i = 0; i < H; ++i) {
    float s = 0.0f;
    for (int j = 0; j < H; ++j) s = fmaf(sp[OW2 + j * H + i], sd2[tid][j], s);
    sd1[tid][i] = sh1[tid][i] > 0.0f ? s : 0.0f;
  }
  __syncthreads();

  // one thread per parameter: its gradient summed over the block's samples
  // in sample order
  float *out = part + (size_t)blockIdx.x * (P + 1);
  for (int p = tid; p <= P; p += CB) {
    float g = 0.0f;
    if (p < OB1) {
      const int j = p / F, f = p - j * F;
      for (int s = 0; s < CB; ++s) g = fmaf(sd1[s][j], sx[s][f], g);
    } else if (p < OW2) {
      const int j = p - OB1;
      for (int s = 0; s < CB; ++s) g += sd1[s][j];
    } else if (p < OB2) {
      const int j = (p - OW2) / H, i = (p - OW2) - j * H;
      for (int s = 0; s < CB; ++s) g = fmaf(sd2[s][j], sh1[s][i], g);
    } else if (p < OW3) {
      const int j = p - OB2;
      for (int s = 0; s < CB; ++s) g += sd2[s][j];
    } else if (p < OB3) {
      const int j = p - OW3;
      for (int s = 0; s < CB; ++s) g = fmaf(sgy[s], sh2[s][j], g);
    } else if (p == OB3) {
      for (int s = 0; s < CB; ++s) g += sgy[s];
    } else {  // p == P: squared residuals
      for (int s = 0; s < CB; ++s) g += sr2[s];
    }
    out[p] = g;
  }
}

// Adds the block sums of each parameter's gradient in block order and
// divides by N.  With m == nullptr it writes the gradient (grad_out) and the
// loss; otherwise it applies one Adam step to params / m / v and writes the
// loss the step started from (loss_out, nullable).
__global__ void cm_update_kernel(const float *__restrict__ part, int nblk, int N,
                                 float *__restrict__ params, float *__restrict__ m,
                                 float *__restrict__ v, float lr, float bc1, float bc2,
                                 float *__restrict__ grad_out, float *__restrict__ loss_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > P) return;
  float g = 0.0f;
  for (int b = 0; b < nblk; ++b) g += part[(size_t)b * (P + 1) + p];
  g /= (float)N;
  if (p == P) {
    if (loss_out) *loss_out = g;
    return;
  }
  if (!m) {
    grad_out[p] = g;
    return;
  }
  constexpr float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  const float mp = beta1 * m[p] + (1.0f - beta1) * g;
  const float vp = beta2 * v[p] + (1.0f - beta2) * g * g;
  m[p] = mp;
  v[p] = vp;
  params[p] -= lr * (mp / bc1) / (sqrtf(vp / bc2) + eps);
}

__global__ void __launch_bounds__(CB) cm_predict_kernel(const float *__restrict__ params,
                                                        const float *__restrict__ feats, int N,
                                                        float *__restrict__ out) {
  __shared__ float sp[P];
  __shared__ float sh1[CB][HS], sh2[CB][HS];
  const int tid = threadIdx.x;
  for (int p = tid; p < P; p += CB) sp[p] = params[p];
  __syncthreads();
  const int64_t n = (int64_t)blockIdx.x * CB + tid;
  if (n >= N) return;
  float x[F];
  for (int f = 0; f < F; ++f) x[f] = feats[n * F + f];
  out[n] = cm_forward(sp, x, sh1[tid], sh2[tid]);
}

}  // namespace

size_t hpc_cm_part_floats(int N) { return (size_t)((N + CB - 1) / CB) * (P + 1); }

int hpc_cm_grad_launch(const hpc_launch &L, const float *params, const float *feats,
                       const float *targets, int N, float *part, float *m, float *v, float lr,
                       float bc1, float bc2, float *grad_out, float *loss_out) {
  const int nblk = (N + CB - 1) / CB;
  cm_grad_kernel<<<nblk, CB, 0, L.stream>>>(params, feats, targets, N, part);
  cm_update_kernel<<<(P + 1 + 255) / 256, 256, 0, L.stream>>>(
      part, nblk, N, m ? const_cast<float *>(params) : nullptr, m, v, lr, bc1, bc2, grad_out,
      loss_out);
  return cudaGetLastError() == cudaSuccess ? HPC_OK : HPC_ERR_CUDA;
}

int hpc_cm_predict_launch(const hpc_launch &L, const float *params, const float *feats, int N,
                          float *out) {
  cm_predict_kernel<<<(N + CB - 1) / CB, CB, 0, L.stream>>>(params, feats, N, out);
  return cudaGetLastError() == cudaSuccess ? HPC_OK : HPC_ERR_CUDA;
}
