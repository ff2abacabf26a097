// Shared definitions of the RI-qsGW CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "molgw_gb300.h"

namespace molgw {

// Launch bookkeeping: every kernel launch of the library goes through KLaunch so
// that the context can count launches and (optionally) time each kernel class
// with CUDA events recorded on the launching stream.
struct KTimer {
  bool enabled = false;
  uint32_t mask = 0;          // kernel classes timed with events
  int64_t launches[MOLGW_K_COUNT] = {0};
  double ms[MOLGW_K_COUNT] = {0};
  int64_t total_launches = 0;
  // pending event pairs, resolved at the next query
  struct Pending { cudaEvent_t a, b; int k; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get_event() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e; cudaEventCreate(&e); return e;
  }
  void resolve() {
    for (auto& p : pending) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ms[p.k] += t;
      pool.push_back(p.a); pool.push_back(p.b);
    }
    pending.clear();
  }
  ~KTimer() {
    for (auto& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct GemmTuner;

// Bounds of the device-side waits and iterations (defaults; molgw_b200_set_wait_limits
// lowers them for the failure-path tests).  A grid barrier polls about 1 s at most.
constexpr long long kGridSpinLimit = 1LL << 24;
constexpr int kBisectRounds = 128;

struct Exec {
  cudaStream_t st = nullptr;
  GemmTuner* tuner = nullptr;  // tile choices of the float64 GEMM (per context), or none
  int* status = nullptr;   // device status word (0 = OK, else a molgw_status)
  KTimer* timer = nullptr;
  bool capturing = false;  // inside stream capture: no events, no allocation
  int coop_cap = 0;        // CTAs a cooperative launch may use (0: the whole device);
                           // concurrent lanes split the device between them
  long long grid_spins = kGridSpinLimit;  // polls of a grid barrier before MOLGW_E_TIMEOUT
  int bisect_rounds = kBisectRounds;      // float64 bisection rounds before MOLGW_E_NOCONV
  int panel_matvec = MOLGW_MATVEC_AUTO;   // mat-vec of the panel kernel with an image arena
};

// Scoped marker: records a start/stop event pair around the kernels launched in
// its lifetime and attributes them to kernel class k.
struct KScope {
  Exec& ex; int k; cudaEvent_t a = nullptr;
  KScope(Exec& e, int kind, int nlaunch = 1) : ex(e), k(kind) {
    if (ex.timer) {
      ex.timer->launches[k] += nlaunch;
      ex.timer->total_launches += nlaunch;
      if (ex.timer->enabled && !ex.capturing && ((ex.timer->mask >> k) & 1u)) {
        a = ex.timer->get_event();
        cudaEventRecord(a, ex.st);
      }
    }
  }
  ~KScope() {
    if (a) {
      cudaEvent_t b = ex.timer->get_event();
      cudaEventRecord(b, ex.st);
      ex.timer->pending.push_back({a, b, k});
    }
  }
};

__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
__host__ __device__ __forceinline__ int ceil_div_d(int a, int b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// Generic strided float64 GEMM: C(i,j) = alpha * sum_k A(i,k) B(k,j) + beta C(i,j)
//   A(i,k) = A[i*sa_m + k*sa_k + b*sa_b], B(k,j) = B[k*sb_k + j*sb_n + b*sb_b],
//   C(i,j) = C[i*sc_m + j*sc_n + b*sc_b], batch index b in [0, batch).
// lower_only computes only the 64x64 output tiles with tile_row >= tile_col.
// ksplit > 1 splits K: partial products go to `work` and are summed in a fixed
// order (deterministic).
// ---------------------------------------------------------------------------
struct GemmF64 {
  int M = 0, N = 0, K = 0, batch = 1;
  const double* A = nullptr; long long sa_m = 0, sa_k = 0, sa_b = 0;
  const double* B = nullptr; long long sb_k = 0, sb_n = 0, sb_b = 0;
  double* C = nullptr; long long sc_m = 0, sc_n = 0, sc_b = 0;
  double alpha = 1.0, beta = 0.0;
  bool lower_only = false;
  int ksplit = 1;
  double* work = nullptr;   // >= ksplit * batch * M * N doubles when ksplit > 1
  int kclass = MOLGW_K_GEMM_F64;  // kernel class for launch accounting
};
void gemm_f64(Exec& ex, const GemmF64& g);

// Measured tile choices of gemm_f64.  Shapes are bucketed (four buckets per octave
// of M, N and K, exact batch and operand layouts); while `active`, a shape not yet
// seen is run once with every tile side (64, 48, 40, 32) into a scratch output
// and the fastest is kept.  All sides give bit-identical results (each output is
// one thread's sequential sum over K), so the choice changes only the time.
struct GemmTuner {
  bool active = false;
  std::vector<std::pair<std::vector<long long>, int>> best;
  double* scratch = nullptr;
  size_t scratch_cap = 0;          // doubles
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int tuned = 0;                   // shapes measured so far
  ~GemmTuner() {
    if (scratch) cudaFree(scratch);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};
// Choose a K split so that the grid fills the GPU; returns 1 if not needed.
int gemm_f64_pick_split(int M, int N, int K, int batch, size_t work_cap_doubles);

// ---------------------------------------------------------------------------
// Float64 symmetric eigensolver (column-major n x n input, lower triangle and
// full 64x64 diagonal tiles used, destroyed).
// ---------------------------------------------------------------------------
struct EigWork {
  int nmax = 0;
  double *d = nullptr, *e = nullptr, *tau = nullptr, *lam = nullptr;
  double *Wp = nullptr;        // n x 64 panel of W (column-major)
  double *part = nullptr;      // partial sums, size part_cap
  size_t part_cap = 0;
  double *scal = nullptr;      // 64 device scalars
  double *S2 = nullptr;        // n x n scratch for the twisted factorisation
  double *Tm = nullptr;        // compact-WY T factors, (nmax/64+1) * 64 * 64
  double *gk = nullptr;        // split-K work for the back-transformation
  size_t gk_cap = 0;
  double *tmp1 = nullptr, *tmp2 = nullptr;  // 64 x ncols_max each
  int ncols_max = 0;
  bool owned = false;          // allocated by eig_work_alloc (freed by eig_work_free)
  // with MOLGW_FLAG_EIG_TC: arena of the 7-digit fixed-point operands of the
  // trailing updates (two fx_mat_bytes(fx_rows, 128, 7)), else nullptr
  void* fx = nullptr;
  long long fx_rows = 0;       // matrices up to fx_rows (n)
  long long fx_cols = 0;       // back-transformations of up to fx_cols columns
  // with MOLGW_FLAG_EIG_TC on the context's own stream: images of the lower 64 x 64
  // tiles of the trailing matrix (eig_sv_bytes(sv_n) bytes) for the panel kernel's
  // fixed-point mat-vec (7-digit BF16 for the tensor cores or 53-bit integers), their
  // scales, the panel's column-maximum partials and the row blocks' scales; else
  // nullptr
  void* sv = nullptr;
  long long sv_n = 0;
};
// Bytes of the fixed-point mat-vec arena for matrices up to n: one 57,344-byte image
// (7 digit planes of 64 x 64 BF16; the integer image takes 32,768) and one scale (or
// exponent) per lower tile, then ceil(n/32) + 2 column-maximum partials, then the
// largest |a| of the integer image.
constexpr long long kSvTileBytes = 7LL * 64 * 64 * 2;
inline long long eig_sv_tiles(long long n) { const long long b = (n + 63) / 64; return b * (b + 1) / 2; }
// Workspace sizes in doubles for matrices up to n and back-transformations of
// up to ncols (>= 64) columns at a time.
constexpr int kMaxPanelGrid = 320;   // CTAs of the tridiagonalisation panel kernel, at most
constexpr size_t kGridBarDoubles = 136; // the panel kernel's barrier block
constexpr size_t eig_part_doubles(size_t n) {
  return 2 * ((n + 31) / 32 + 1) + ((n + 31) / 32 + 1) * 128 + 128 + 2 * n * 128 + kGridBarDoubles +
         ((n + 63) / 64) * ((n + 63) / 64 + 1) / 2 * 64 + (size_t)kMaxPanelGrid * n + 64;
}
constexpr size_t eig_gk_doubles(size_t n, size_t ncols) {
  return (16 * 64 * ncols > 8 * (n / 64 + 1) * 64 * 64) ? 16 * 64 * ncols : 8 * (n / 64 + 1) * 64 * 64;
}
inline size_t eig_sv_bytes(long long n) {
  return (size_t)(eig_sv_tiles(n) * (kSvTileBytes + 8) + ((n + 31) / 32 + 2) * 8 + 8 + 256);
}
constexpr size_t eig_work_doubles(size_t n, size_t ncols) {
  return 4 * n + n * 64 + eig_part_doubles(n) + 64 + n * n + 2 * (n / 64 + 1) * 64 * 64 + 2 * 64 * ncols +
         eig_gk_doubles(n, ncols);
}
// Lay an EigWork out over caller-provided device memory of eig_work_doubles(n, ncols) doubles.
void eig_work_carve(EigWork& w, double* base, int nmax, int ncols_max);
int eig_work_alloc(EigWork& w, int nmax, int ncols_max);
void eig_work_free(EigWork& w);

// CTAs of the persistent panel kernel that are co-resident on the device.
int tridiag_coop_capacity();
// Reduce A (column-major, ld = n) to tridiagonal T = Q^T A Q (d, e), keeping the
// Householder vectors in A (column i, rows i+1.., unit at row i+1 made explicit,
// zeros above) and tau.
void tridiagonalize(Exec& ex, EigWork& w, int n, double* A);
// Eigenvalues of T ascending into w.lam (bisection on Sturm counts).
void tridiag_eigvals(Exec& ex, EigWork& w, int n);
// Eigenvectors of T by twisted factorisations: ZT[j*ldz + s] = component j of vector s.
void tridiag_eigvecs(Exec& ex, EigWork& w, int n, double* ZT, long long ldz);
// Compact-WY T factors of every 64-column panel of the Householder vectors in A.
void build_wy(Exec& ex, EigWork& w, int n, const double* A);
// X (n x ncols, element (r, c) at X[r*sr + c*sc]) <- Q^T X (trans = 1) or Q X (trans = 0).
void apply_q(Exec& ex, EigWork& w, int n, const double* A, double* X, long long sr, long long sc,
             int ncols, int trans);

}  // namespace molgw
