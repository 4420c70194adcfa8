// fe_noalloc.cu -- y = K x without allocating device memory during the call.
//
// fe_spmv converts x into the SpMV's input precision in a buffer it
// allocates on first use.  fe_spmv_noalloc stages that converted input in a
// fixed array owned by this file instead, so the call itself never
// allocates.  The paper has no counterpart: this serves callers that must not
// allocate while they run (see include/fe.h).
//
// With CUDA's lazy module loading, the array below gets its device memory
// when this file's module is first loaded, which happens at the first use of
// anything in it (the symbol lookup or a kernel launch), and each kernel's
// code is placed in device memory at its first launch.  fe_mesh_create
// therefore calls fe_noalloc_prepare, which does all of that on the mesh's
// device while allocating is still allowed: it looks the array's address up,
// loads the staging kernels and every SpMV kernel.  A later fe_spmv_noalloc
// call only reads the cached address and launches loaded kernels.
#include <mutex>

#include "fe_internal.h"

// 2^20 FP64 entries (8 MiB): the largest ndof the entry point accepts.  An
// FP32 input uses the first half of the bytes.  Every GPU that loads the
// library holds this array until the process exits.
static constexpr int64_t kNoAllocMaxDof = int64_t(1) << 20;
static __device__ __align__(256) double g_spmv_input[kNoAllocMaxDof];

// Device address of g_spmv_input, looked up once per device (in host code the
// symbol's name is only a host-side stand-in, not a device address).
static constexpr int kMaxDevices = 64;
static std::mutex g_addr_mu;
static void* g_addr[kMaxDevices] = {};

template <class T>
__global__ void k_stage_input(int64_t n, const double* __restrict__ x, T* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (T)x[i];
}

// `device` must be current.  load = true: look the address up if this device
// has none yet (loads the module); false: only read the cached address.
static int input_array(int device, bool load, void** out) {
  if (device < 0 || device >= kMaxDevices) return fe_set_error("device ordinal %d out of range", device), FE_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[device]) {
    if (!load)
      return fe_set_error("the fixed SpMV input array of device %d was not prepared by fe_mesh_create", device),
             FE_ERR_STATE;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_spmv_input);
    if (e != cudaSuccess || !p) {
      fe_set_error("cudaGetSymbolAddress for the fixed SpMV input array failed: %s", cudaGetErrorString(e));
      return FE_ERR_CUDA;
    }
    g_addr[device] = p;
  }
  *out = g_addr[device];
  return FE_OK;
}

int fe_noalloc_prepare(fe_mesh m) {
  void* input = nullptr;
  FE_TRY(input_array(m->device, true, &input));
  cudaFuncAttributes a;
  FE_CUDA(cudaFuncGetAttributes(&a, (const void*)k_stage_input<double>));
  FE_CUDA(cudaFuncGetAttributes(&a, (const void*)k_stage_input<float>));
  return fe_spmv_preload(m);
}

extern "C" int fe_spmv_noalloc(fe_mesh m, const double* x, double* y) {
  if (!m || !x || !y) return fe_set_error("NULL argument"), FE_ERR_ARG;
  if (m->ndof > kNoAllocMaxDof)
    return fe_set_error("fe_spmv_noalloc accepts at most %lld unknowns (mesh has %lld); use fe_spmv",
                        (long long)kNoAllocMaxDof, (long long)m->ndof),
           FE_ERR_ARG;
  if (m->prec < 0) return fe_set_error("no tangent assembled"), FE_ERR_STATE;
  FE_CUDA(cudaSetDevice(m->device));
  void* input = nullptr;
  FE_TRY(input_array(m->device, false, &input));
  // the whole input range is overwritten by every call: nothing to clear
  const unsigned grid = (unsigned)((m->ndof + 255) / 256);
  if (m->prec == FE_PREC_FP64)
    k_stage_input<double><<<grid, 256, 0, m->stream>>>(m->ndof, x, (double*)input);
  else
    k_stage_input<float><<<grid, 256, 0, m->stream>>>(m->ndof, x, (float*)input);
  FE_CUDA(cudaGetLastError());
  FE_TRY(fe_spmv_from_input(m, input, y));
  return fe_check_device_error(m);
}
