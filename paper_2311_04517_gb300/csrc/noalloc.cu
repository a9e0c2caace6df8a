// Allocation-free full-data objective.
//
// Some callers cannot allocate device memory at the moment they need the
// objective: code running while a CUDA stream is being captured into a graph
// (cudaMalloc is not allowed there), real-time loops whose memory budget is
// fixed up front, or hosts that hand out device memory only through their
// own pool.  hpc_objective_noalloc serves them: it needs no context and
// allocates nothing.  The per-block partial sums and the completion counter
// of the objective kernel live in the file-scope array below instead of a
// context's scratch.
//
// Limits and sharing rules:
//  - the array holds HPC_NOALLOC_MAX_BLOCKS partial sums plus a counter
//    (about 16 KB); it is part of the library image, so every GPU that loads
//    the library keeps it until the process exits;
//  - every call on a device uses the same array and leaves its last contents
//    there, so calls that may overlap on the GPU (different streams, or
//    several host threads) race and give wrong results: serialise them;
//  - a call made while its stream is not being captured looks the array's
//    device address up again (cudaGetSymbolAddress, with the call's device
//    current), so a context reset between calls is harmless; a call made
//    while its stream is being captured into a graph reuses the address the
//    latest uncaptured call on that device found, so make one uncaptured
//    call on each device first, with the same padded dimension and the same
//    k class (k <= 32 or k > 32) as the captured call: that first call also
//    loads the kernel and sets its shared-memory limit, neither of which
//    should happen inside a capture.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

#define HPC_NOALLOC_MAX_BLOCKS 2048
#define HPC_NOALLOC_MAX_DEVICES 64

namespace {

// [0, MAX_BLOCKS) doubles: per-block partial objectives; then one unsigned
// completion counter (must be zero when a launch starts).
static __device__ __align__(256) double g_noalloc_scratch[HPC_NOALLOC_MAX_BLOCKS + 32];

std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[HPC_NOALLOC_MAX_DEVICES];

// Device address of the array on the current device: looked up afresh when
// `stream` is not being captured, else the one the latest uncaptured call
// found (a capture must not trigger the lookup).
int noalloc_scratch(int device, cudaStream_t stream, void **out) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    return HPC_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (cs == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return HPC_ERR_CUDA;
    }
    g_noalloc_ptr[device] = p;
  } else if (!g_noalloc_ptr[device]) {
    return HPC_ERR_ARG;  // no uncaptured call on this device yet
  }
  *out = g_noalloc_ptr[device];
  return HPC_OK;
}

}  // namespace

extern "C" int hpc_objective_noalloc(const float *X, int64_t n, int32_t d, const float *C,
                                     int32_t k, const uint8_t *degenerate, double *f_out,
                                     int32_t *labels_out, int32_t *status_out, void *stream) {
  if (d < 1 || d > HPC_MAX_D || n < 0 || k < 1 || !C || !f_out || !status_out || (n > 0 && !X))
    return HPC_ERR_ARG;
  if ((X && ((uintptr_t)X & 15u)) || ((uintptr_t)C & 15u)) return HPC_ERR_ARG;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= HPC_NOALLOC_MAX_DEVICES) {
    cudaGetLastError();
    return HPC_ERR_CUDA;
  }
  void *scratch = nullptr;
  if (int rc = noalloc_scratch(device, (cudaStream_t)stream, &scratch)) return rc;
  hpc_launch L;
  L.stream = (cudaStream_t)stream;
  if (cudaDeviceGetAttribute(&L.num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&L.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
          cudaSuccess)
    return HPC_ERR_CUDA;
  L.smem_optin -= 2048;
  double *part = static_cast<double *>(scratch);
  unsigned *counter = reinterpret_cast<unsigned *>(part + HPC_NOALLOC_MAX_BLOCKS);
  // what must start at zero: the completion counter and the caller's status
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned), L.stream) != cudaSuccess ||
      cudaMemsetAsync(status_out, 0, sizeof(int32_t), L.stream) != cudaSuccess)
    return HPC_ERR_CUDA;
  ObjArgsHost h{};
  h.X = X;
  h.n = n;
  h.d = d;
  h.k = k;
  h.C = C;
  h.deg = degenerate;
  h.f_out = f_out;
  h.labels = labels_out;
  h.status = status_out;
  h.part = part;
  h.done_count = counter;
  h.max_blocks = HPC_NOALLOC_MAX_BLOCKS;  // grid never exceeds the partial sums held
  return hpc_objective_launch(L, h);
}
