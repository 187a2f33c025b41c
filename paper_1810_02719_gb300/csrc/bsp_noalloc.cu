// Allocation-free orthonormalisation of one block: the fused CholeskyQR2
// kernel with its scratch in a fixed static device array instead of a
// library-allocated workspace.
//
// Who needs it: callers that may not allocate device memory while they run,
// for instance a streaming pipeline that orthonormalises submeshes as a
// scanner delivers them and must keep its per-call latency bounded (a
// cudaMalloc can synchronise the whole device and take unbounded time), or a
// host application whose device memory is owned by another allocator and must
// not grow behind its back.  They pass their own input and output buffers; the
// only other memory used is the static array below.
#include <mutex>
#include <string>

#include "bsp_internal.cuh"

namespace {

// Largest block this entry point accepts.
constexpr int kMaxRows = 2048;
constexpr int kMaxCols = 64;
constexpr int kMaxPanels = 8;   // cluster size of the fused kernel
constexpr int kMeta = 64;       // int32 slots: batch list, block pointers, widths, status

// Scratch: metadata, then the partial Grams of every panel, then the summed
// Gram.  Every GPU that loads this library holds it until the process exits.
constexpr size_t kGramFloats = (size_t)kMaxPanels * kMaxCols * kMaxCols + (size_t)kMaxCols * kMaxCols;
constexpr size_t kScratchBytes = kMeta * sizeof(int32_t) + kGramFloats * sizeof(float);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int noalloc_fail(int code, const char* msg) {
  bsp::set_last_error(msg);
  return code;
}

// True when p is device (or managed) memory of device `dev`: a host buffer or
// another GPU's buffer would reach the kernel as a bad device address.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) &&
         at.device == dev;
}

}  // namespace

extern "C" int bsp_onorm_noalloc(const float* Y, float* Q, int32_t n, int32_t c, void* stream) {
  bsp::set_last_error("");
  if (!Y || !Q) return noalloc_fail(BSP_ERR_INVALID_ARG, "Y and Q are required");
  if (n < 1 || c < 1 || c > n) return noalloc_fail(BSP_ERR_INVALID_ARG, "need 1 <= c <= n");
  if (n > kMaxRows || c > kMaxCols)
    return noalloc_fail(BSP_ERR_INVALID_ARG,
                        "bsp_onorm_noalloc accepts at most 2048 rows and 64 columns");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return noalloc_fail(BSP_ERR_CUDA, "no usable current CUDA device");
  }
  if (!on_device(Y, dev) || !on_device(Q, dev))
    return noalloc_fail(BSP_ERR_INVALID_ARG,
                        "Y and Q must be device memory of the current CUDA device");
  // One-time set-up per device, with that device current: the device address
  // of the static scratch array (its name is only a host stand-in here).
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return noalloc_fail(BSP_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
      }
      bsp::configure_fused_kernels();
      cudaGetLastError();
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* meta = static_cast<int32_t*>(base);
  float* gram = reinterpret_cast<float*>(meta + kMeta);
  // batch = {0}, block pointers = {0, n}, width = {c}; status word cleared
  const int32_t host_meta[5] = {0, 0, n, c, 0};
  if (cudaMemcpyAsync(meta, host_meta, sizeof(host_meta), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(BSP_ERR_CUDA, "copy of the call's parameters failed");
  }
  bsp::DenseArgs a{meta + 0, 1, meta + 1, meta + 3, c, c, n, meta + 4};
  int rc = bsp::launch_cholqr2_fused<float, float>(a, Y, Q, gram, kMaxPanels, s, 2);
  if (rc != BSP_OK) {
    cudaGetLastError();
    return noalloc_fail(rc == BSP_ERR_INVALID_ARG ? BSP_ERR_INVALID_ARG : BSP_ERR_CUDA,
                        "launch of the orthonormalisation kernel failed");
  }
  int32_t status = 0;
  if (cudaMemcpyAsync(&status, meta + 4, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(BSP_ERR_CUDA, "CUDA error while orthonormalising");
  }
  if (status & bsp::ST_NUMERICAL)
    return noalloc_fail(BSP_ERR_NUMERICAL, "Gram matrix not positive definite or non-finite");
  return BSP_OK;
}
