// Forward power evaluation that performs no device allocation.
//
// dpf_power_noalloc computes S_calc = V (Y V)^* (FP64) like dpf_power, but
// instead of a workspace it uses one fixed scratch array that is part of the
// library image: a file-scope __device__ array of DPF_NOALLOC_MAX_ELEMS
// complex values (4 MiB).  Every GPU that loads the library holds this array
// until the process exits, whether or not the entry point is used.
//
// Some callers cannot call cudaMalloc at all: code that runs inside a host
// application which owns the whole device memory budget through its own pool
// (a raw cudaMalloc there fails or escapes the application's accounting), and
// latency-critical loops where the implicit device synchronisation of
// cudaMalloc/cudaFree is not acceptable.  They can still evaluate the power
// balance through this entry point, given a Y_bus built beforehand.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "dpf_internal.h"

namespace {

constexpr int kMaxDevices = 64;

// The scratch: V = |V| e^{j theta} of every (case, bus), case-major.
static __device__ __align__(256) double2 g_noalloc_v[DPF_NOALLOC_MAX_ELEMS];

// Device address of g_noalloc_v, one per device (host code cannot use the
// symbol's name as a device pointer).  Looked up on the first call on each
// device and kept for the life of the process: a cudaDeviceReset destroys the
// context the address belongs to, so the entry point must not be used on a
// device after it has been reset.
double2* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(double2** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return dpf::fail(DPF_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return dpf::fail(DPF_E_UNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_v);
    if (e != cudaSuccess || !p)
      return dpf::fail(DPF_E_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = (double2*)p;
  }
  *out = g_scratch_ptr[dev];
  return DPF_OK;
}

// V of internal row i of case k from the caller's case-major user-order inputs.
__global__ void k_na_volt(const double* __restrict__ va, const double* __restrict__ vm,
                          const int32_t* __restrict__ perm, int N, int K, double2* __restrict__ V) {
  const size_t n = (size_t)N * K;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / N), i = (int)(e % N);
    const size_t u = (size_t)k * N + perm[i];
    double s, c;
    sincos(va[u], &s, &c);
    V[e] = make_double2(vm[u] * c, vm[u] * s);
  }
}

// S_i = V_i conj(sum_j Y_ij V_j), written back in user bus order.
__global__ void k_na_power(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double2* __restrict__ val, const int32_t* __restrict__ perm, int N, int K,
                           const double2* __restrict__ V, double* __restrict__ p_out, double* __restrict__ q_out) {
  const size_t n = (size_t)N * K;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / N), i = (int)(e % N);
    const double2* Vk = V + (size_t)k * N;
    double ir = 0.0, ii = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      const double2 y = val[p], v = Vk[col[p]];
      ir = fma(y.x, v.x, fma(-y.y, v.y, ir));
      ii = fma(y.x, v.y, fma(y.y, v.x, ii));
    }
    const double2 vi = Vk[i];
    const size_t u = (size_t)k * N + perm[i];
    if (p_out) p_out[u] = vi.x * ir + vi.y * ii;
    if (q_out) q_out[u] = vi.y * ir - vi.x * ii;
  }
}

}  // namespace

extern "C" int dpf_power_noalloc(const dpf_ybus* y, int32_t n_case, const double* va, const double* vm,
                                 double* p_calc, double* q_calc, void* stream) {
  dpf::clear_error();
  if (!y || !va || !vm) return dpf::fail(DPF_E_INVALID, "dpf_power_noalloc: NULL argument");
  if (!y->dev.ready) return dpf::fail(DPF_E_STATE, "Y_bus is not on the device (dpf_ybus_upload)");
  if (n_case < 1) return dpf::fail(DPF_E_INVALID, "n_case must be >= 1");
  const long long elems = (long long)n_case * y->n;
  if (elems > DPF_NOALLOC_MAX_ELEMS)
    return dpf::fail(DPF_E_INVALID,
                     "dpf_power_noalloc: n_case * n_bus = %lld exceeds the fixed scratch of %d elements",
                     elems, DPF_NOALLOC_MAX_ELEMS);
  int dev = -1;
  const cudaError_t ge = cudaGetDevice(&dev);
  if (ge != cudaSuccess) return dpf::fail(DPF_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(ge));
  if (dev != y->dev.device)
    return dpf::fail(DPF_E_STATE, "current device %d differs from the Y_bus device %d", dev, y->dev.device);
  double2* V = nullptr;
  const int rc = scratch_for_current_device(&V);
  if (rc != DPF_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int threads = 256;
  const int blocks = (int)std::min<long long>((elems + threads - 1) / threads, 152LL * 16);
  // V is written in full by k_na_volt before k_na_power reads it; nothing in
  // the scratch needs to start at zero.
  k_na_volt<<<blocks, threads, 0, s>>>(va, vm, y->dev.perm, y->n, n_case, V);
  k_na_power<<<blocks, threads, 0, s>>>(y->dev.row_ptr, y->dev.col, y->dev.val64, y->dev.perm, y->n, n_case, V,
                                        p_calc, q_calc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dpf::fail(DPF_E_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return DPF_OK;
}
