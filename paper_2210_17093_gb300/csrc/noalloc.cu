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
// The array is sized for n <= MOLGW_NOALLOC_NMAX (256): 634,042 doubles
// (5.07 MB, the status slot included), held by every GPU that loads the library
// until the process exits.
#include <cuda.h>

#include "stages.cuh"

namespace {

constexpr size_t kNMax = MOLGW_NOALLOC_NMAX;
constexpr size_t kStatusDoubles = 32;          // 256 bytes, keeps what follows aligned
constexpr size_t kScratchDoubles = kStatusDoubles + kNMax * kNMax + molgw::eig_work_doubles(kNMax, kNMax);
static_assert(kScratchDoubles == 634042, "the workspace size stated in the header and this file's preamble");

constexpr int kMaxDevices = 64;
// Device address of the array, per device, and the id of the CUDA context it was
// looked up in (a context created after cudaDeviceReset gets a new id, and the
// module holding the array a new address).
struct ScratchAddr { double* ptr; unsigned long long ctx_id; };
ScratchAddr g_scratch_addr[kMaxDevices] = {};

}  // namespace

// The scratch itself.  In host code `g_noalloc_scratch` is only a host-side
// stand-in for the symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

namespace {

// Id of the CUDA context current on this thread (0 if there is none yet, or if the
// driver does not offer the calls).  The driver functions are looked up through the
// runtime, so that the library loads on machines without a driver.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
      cudaGetLastError();
      return 0;
    }
    get_current = (CtxGetCurrentFn)f1;
    get_id = (CtxGetIdFn)f2;
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c) return 0;
  if (get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Set-up, once per device (again only if the device's context was replaced), with
// that device current: look up the array's device address.
int scratch_for_current_device(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return MOLGW_E_CUDA;
  unsigned long long id = current_ctx_id();
  ScratchAddr& s = g_scratch_addr[dev];
  if (!s.ptr || id == 0 || s.ctx_id != id) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return MOLGW_E_CUDA;
    }
    if (id == 0) id = current_ctx_id();   // the lookup created the primary context
    s.ptr = p;
    s.ctx_id = id;
  }
  *out = s.ptr;
  return MOLGW_OK;
}

// Device (or managed) memory that belongs to device `dev`.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" int molgw_b200_eigh_noalloc(int n, const double* A, double* w, double* Z, void* stream) {
  if (n < 1 || n > (int)kNMax || !A || !w) return MOLGW_E_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MOLGW_E_CUDA;
  }
  if (!on_device(A, dev) || !on_device(w, dev) || (Z && !on_device(Z, dev))) return MOLGW_E_ARG;
  double* base = nullptr;
  int r = scratch_for_current_device(dev, &base);
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
