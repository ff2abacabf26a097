// Allocation-free variant of the float64 symmetric eigensolver (molgw_b200_eigh).
//
// Some callers cannot allocate device memory at the point where they need an
// eigendecomposition: an application that hands all device memory to its own
// pool allocator and forbids other allocations, a latency-bound loop that must
// not pay for cudaMalloc or for the device-wide synchronisation of cudaFree,
// or a plug-in that runs when the host program has already claimed the memory
// it is allowed to use.  molgw_b200_eigh_noalloc serves them: every buffer the
// solver needs (the working copy of A, the tridiagonal factors, the Householder
// panel, partial sums, compact-WY factors, split-K partials and the status word)
// lives in one file-scope device array of fixed size, so the call allocates
// nothing.  The caller passes device pointers for the input and the outputs.
//
// The array is sized for n <= MOLGW_NOALLOC_NMAX (256): 633,914 doubles
// (5.07 MB, the status slot included), held by every GPU that loads the library
// until the process exits.
#include "stages.cuh"

namespace {

constexpr size_t kNMax = MOLGW_NOALLOC_NMAX;
constexpr size_t kStatusDoubles = 32;          // 256 bytes, keeps what follows aligned
constexpr size_t kScratchDoubles = kStatusDoubles + kNMax * kNMax + molgw::eig_work_doubles(kNMax, kNMax);

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};   // device address of the array, per device

}  // namespace

// The scratch itself.  In host code `g_noalloc_scratch` is only a host-side
// stand-in for the symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

namespace {

// Once per device, with that device current: look up the array's device address.
int scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return MOLGW_E_CUDA;
  }
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return MOLGW_E_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return MOLGW_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int molgw_b200_eigh_noalloc(int n, const double* A, double* w, double* Z, void* stream) {
  if (n < 1 || n > (int)kNMax || !A || !w) return MOLGW_E_ARG;
  if (!on_device(A) || !on_device(w) || (Z && !on_device(Z))) return MOLGW_E_ARG;
  double* base = nullptr;
  int r = scratch_for_current_device(&base);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  int* status = (int*)base;
  double* Acopy = base + kStatusDoubles;
  molgw::EigWork ew;
  molgw::eig_work_carve(ew, Acopy + kNMax * kNMax, (int)kNMax, (int)kNMax);
  molgw::Exec ex;
  ex.st = st;
  ex.status = status;
  ex.timer = nullptr;
  // the array keeps the previous call's contents: only the status word must start at zero
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) { cudaGetLastError(); return MOLGW_E_CUDA; }
  if (cudaMemcpyAsync(Acopy, A, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return MOLGW_E_CUDA;
  }
  molgw::eigh_dense(ex, ew, n, Acopy, Z);
  if (cudaMemcpyAsync(w, ew.lam, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return MOLGW_E_CUDA;
  }
  if (cudaGetLastError() != cudaSuccess) return MOLGW_E_CUDA;
  int h_status = 0;
  if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return MOLGW_E_CUDA;
  }
  return h_status;
}
