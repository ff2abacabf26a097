// Float64 Householder tridiagonalisation of a symmetric matrix on the GPU.
//
// Blocked one-stage reduction in the manner of LAPACK's dsytrd/dlatrd (lower
// triangle): 64-column panels; within a panel each column i gets
//   K1  the deferred updates of the panel's earlier reflectors (rows i..n-1),
//       plus the partial sums of squares of the part to annihilate;
//   K2  the reflector H_i = I - tau v v^T (beta, tau, v scaled in place);
//   K3  y = A22 v over the not-yet-updated trailing matrix, 64x64 tiles, the
//       lower triangle read once per use (transposed tiles for the upper half),
//       partial sums per tile chunk (deterministic), plus V^T v and W^T v;
//   K4  the W column w = tau (y - W V^T v - V W^T v) and the partials of w^T v;
// the rank-1 correction w += -tau/2 (w^T v) v of column i is applied by the
// next column's K1 (or K5 at the end of the panel).  After the panel the
// trailing matrix gets A -= V W^T + W V^T as one GEMM with K = 128 over the
// lower 64x64 tiles (diagonal tiles in full).
//
// Storage: A column-major, ld = n.  Every 64x64 diagonal tile is kept full
// (both halves); off-diagonal tiles only below the diagonal.  The upper tiles
// are never read.
//
// On GB300 the FP64 pipe (~2 DFMA/clk/SM) rather than HBM bounds both the
// symmetric matrix-vector products (2 flops per 8-byte element) and the
// rank-2k updates, so the kernels spread every FP64 loop over the whole GPU.
#include <algorithm>

#include "common.cuh"

namespace molgw {

namespace {

constexpr int NBP = 64;     // panel width
constexpr int TB = 64;      // tile size of the symmetric matrix-vector product
constexpr int TPC = 8;      // tiles per CTA in K3
constexpr int RT = 256;     // rows per CTA in K1/K2/K4

struct TriParams {
  int n, i, k0, j;          // column, panel start, index in panel
  double* A;
  double* Wp;               // n x NBP, column-major
  double* d; double* e; double* tau;
  double* scal;
  double* p_ss; int n_ss;   // K1 sum-of-squares partials
  double* p_vw;             // K3: per row block, 2*NBP values (V^T v, W^T v)
  double* p_y;              // K3: nchunk x n
  double* p_wv; int n_wv;   // K4: w^T v partials; n_wv_prev for the previous column
  int n_wv_prev;
  int rb0, nrb, nchunk;     // K3 geometry
};

__device__ __forceinline__ double blk_reduce_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// Sum of `cnt` partials, computed by every thread of the block (same order).
__device__ double sum_partials(const double* p, int cnt, double* sh) {
  double v = 0.0;
  for (int k = threadIdx.x; k < cnt; k += blockDim.x) v += p[k];
  double s = blk_reduce_sum(v, sh);
  __syncthreads();
  if (threadIdx.x == 0) sh[32] = s;
  __syncthreads();
  return sh[32];
}

// K1: column update of column i with the panel's earlier reflectors.
__global__ void __launch_bounds__(RT) k1_col_update(TriParams p) {
  __shared__ double sh[40];
  __shared__ double Wi[NBP], Vi[NBP];
  const int n = p.n, i = p.i, j = p.j;
  const long long ld = n;
  double* A = p.A;
  double alpha_w = 0.0;
  if (j > 0) {
    // correction of the previous column's W: alpha_w = -tau/2 * w^T v
    const double s = sum_partials(p.p_wv, p.n_wv_prev, sh);
    alpha_w = -0.5 * p.tau[i - 1] * s;
  }
  for (int c = threadIdx.x; c < j; c += blockDim.x) {
    double w = p.Wp[i + (long long)c * ld];
    if (c == j - 1) w = p.scal[3] + alpha_w;   // uncorrected W[i, j-1] from the slot (v_{i-1}[i] = 1)
    Wi[c] = w;
    Vi[c] = A[i + (long long)(p.k0 + c) * ld];
  }
  __syncthreads();
  const int r = i + blockIdx.x * RT + threadIdx.x;
  double sq = 0.0;
  if (r < n) {
    if (j > 0) {
      double* wc = p.Wp + r + (long long)(j - 1) * ld;
      const double vprev = A[r + (long long)(i - 1) * ld];
      *wc = *wc + alpha_w * vprev;
    }
    double a = A[r + (long long)i * ld];
    for (int c = 0; c < j; ++c) {
      const double vr = A[r + (long long)(p.k0 + c) * ld];
      const double wr = p.Wp[r + (long long)c * ld];
      a -= vr * Wi[c] + wr * Vi[c];
    }
    A[r + (long long)i * ld] = a;
    if (r == i) p.d[i] = a;
    if (r == i + 1) p.scal[0] = a;
    if (r >= i + 2) sq = a * a;
  }
  const double s = blk_reduce_sum(sq, sh);
  if (threadIdx.x == 0) p.p_ss[blockIdx.x] = s;
}

// K2: Householder reflector (LAPACK dlarfg convention, beta = -sign(alpha) ||x||).
__global__ void __launch_bounds__(RT) k2_householder(TriParams p) {
  __shared__ double sh[40];
  const int n = p.n, i = p.i;
  const long long ld = n;
  const double sumsq = sum_partials(p.p_ss, p.n_ss, sh);
  const double alpha = p.scal[0];
  double tau = 0.0, beta = alpha, scale = 0.0;
  if (sumsq > 0.0) {
    const double nrm = sqrt(alpha * alpha + sumsq);
    beta = (alpha >= 0.0) ? -nrm : nrm;
    tau = (beta - alpha) / beta;
    scale = 1.0 / (alpha - beta);
  }
  const int r = i + 2 + blockIdx.x * RT + threadIdx.x;
  if (r < n) {
    double* a = p.A + r + (long long)i * ld;
    *a = (*a) * scale;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    p.e[i] = beta;
    p.tau[i] = tau;
    p.scal[1] = tau;
    p.A[(i + 1) + (long long)i * ld] = 1.0;
  }
}

// K3: partial y = A22 v for row block R over a chunk of column blocks.
__global__ void __launch_bounds__(256) k3_symv(TriParams p) {
  __shared__ double tile[TB * (TB + 1)];
  __shared__ double vJ[TB];
  __shared__ double red[4][TB];
  const int n = p.n, i = p.i;
  const long long ld = n;
  const int R = p.rb0 + blockIdx.x / p.nchunk;
  const int chunk = blockIdx.x % p.nchunk;
  const int J0 = p.rb0 + chunk * TPC;
  const int J1 = min(p.rb0 + p.nrb, J0 + TPC);
  const int t = threadIdx.x;
  const int lo = i + 1;                         // first row/column of A22
  const double* A = p.A;
  const double* v = p.A + (long long)i * ld;    // v[r] for r >= i+1 (unit at i+1)
  double acc = 0.0;                             // this thread's partial for y[R*TB + t%64]
  for (int J = J0; J < J1; ++J) {
    __syncthreads();
    if (t < TB) {
      const int r = J * TB + t;
      vJ[t] = (r >= lo && r < n) ? v[r] : 0.0;
    }
    // load the stored tile: rows of the lower block, columns of the upper one
    const int tr = (J >= R) ? J : R, tc = (J >= R) ? R : J;  // tile (tr, tc) has tr >= tc
    for (int k = 0; k < 16; ++k) {
      const int rr = t % TB, cc = t / TB + 4 * k;
      const int gr = tr * TB + rr, gc = tc * TB + cc;
      tile[cc * (TB + 1) + rr] = (gr < n && gc < n) ? A[gr + (long long)gc * ld] : 0.0;
    }
    __syncthreads();
    const int q = t / TB, x = t % TB;
    double s = 0.0;
    if (J <= R) {       // y[R*TB + x] += sum_c tile(x, c) vJ[c]  (J == R: full diagonal tile)
      for (int c = q * 16; c < q * 16 + 16; ++c) s += tile[c * (TB + 1) + x] * vJ[c];
    } else {            // y[R*TB + x] += sum_r tile(r, x) vJ[r]  (tile is block (J, R))
      for (int r = q * 16; r < q * 16 + 16; ++r) s += tile[x * (TB + 1) + r] * vJ[r];
    }
    acc += s;
  }
  __syncthreads();
  red[t / TB][t % TB] = acc;
  __syncthreads();
  if (t < TB) {
    const int r = R * TB + t;
    const double y = red[0][t] + red[1][t] + red[2][t] + red[3][t];
    if (r < n) p.p_y[(long long)chunk * n + r] = y;
  }
  // V^T v and W^T v partials over this row block (chunk 0 only)
  if (chunk == 0) {
    const int j = p.j;
    for (int c = t; c < 2 * j; c += blockDim.x) {
      const int cc = (c < j) ? c : c - j;
      double s = 0.0;
      for (int rr = 0; rr < TB; ++rr) {
        const int r = R * TB + rr;
        if (r < lo || r >= n) continue;
        const double vr = v[r];
        const double m = (c < j) ? A[r + (long long)(p.k0 + cc) * ld] : p.Wp[r + (long long)cc * ld];
        s += m * vr;
      }
      p.p_vw[(long long)(R - p.rb0) * (2 * NBP) + c] = s;
    }
  }
}

// K4: W column j = tau (y - W vtv - V wtv), partials of w^T v.
__global__ void __launch_bounds__(RT) k4_wcol(TriParams p) {
  __shared__ double sh[40];
  __shared__ double vtv[NBP], wtv[NBP];
  const int n = p.n, i = p.i, j = p.j;
  const long long ld = n;
  for (int c = threadIdx.x; c < 2 * j; c += blockDim.x) {
    double s = 0.0;
    for (int R = 0; R < p.nrb; ++R) s += p.p_vw[(long long)R * (2 * NBP) + c];
    if (c < j) vtv[c] = s; else wtv[c - j] = s;
  }
  __syncthreads();
  const double tau = p.scal[1];
  const int r = i + 1 + blockIdx.x * RT + threadIdx.x;
  double part = 0.0;
  if (r < n) {
    double y = 0.0;
    for (int c = 0; c < p.nchunk; ++c) y += p.p_y[(long long)c * n + r];
    for (int c = 0; c < j; ++c) {
      y -= p.Wp[r + (long long)c * ld] * vtv[c];
      y -= p.A[r + (long long)(p.k0 + c) * ld] * wtv[c];
    }
    const double w = tau * y;
    p.Wp[r + (long long)j * ld] = w;
    if (r == i + 1) p.scal[3] = w;
    part = w * p.A[r + (long long)i * ld];
  }
  const double s = blk_reduce_sum(part, sh);
  if (threadIdx.x == 0) p.p_wv[blockIdx.x] = s;
}

// K5: W[:, j] += alpha_w v at the end of a panel; packs [V W] and [W V] for the update.
__global__ void __launch_bounds__(RT) k5_finish(TriParams p, int nbp, int k1, double* VW, double* WV) {
  __shared__ double sh[40];
  const int n = p.n, i = p.i, j = p.j;
  const long long ld = n;
  const double s = sum_partials(p.p_wv, p.n_wv, sh);
  const double alpha_w = -0.5 * p.tau[i] * s;
  const int r = i + 1 + blockIdx.x * RT + threadIdx.x;
  if (r < n) {
    double* wc = p.Wp + r + (long long)j * ld;
    *wc = *wc + alpha_w * p.A[r + (long long)i * ld];
  }
  // pack rows r >= k1 (grid covers rows i+1 .. n-1 and i+1 <= k1)
  if (r >= k1 && r < n) {
    const long long m = n - k1;
    const long long rr = r - k1;
    for (int c = 0; c < nbp; ++c) {
      const double vv = p.A[r + (long long)(p.k0 + c) * ld];
      const double ww = p.Wp[r + (long long)c * ld];
      VW[rr + (long long)c * m] = vv;
      VW[rr + (long long)(nbp + c) * m] = ww;
      WV[rr + (long long)c * m] = ww;
      WV[rr + (long long)(nbp + c) * m] = vv;
    }
  }
}

__global__ void k_last_diag(double* A, int n, double* d) {
  if (threadIdx.x == 0 && blockIdx.x == 0) d[n - 1] = A[(n - 1) + (long long)(n - 1) * n];
}

// Zero everything on or above the diagonal of column c (c < n-1) so that column
// c is exactly the Householder vector v_c (unit at row c+1); column n-1 is zeroed.
__global__ void k_clean(double* A, int n) {
  const long long total = (long long)n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx % n), c = (int)(idx / n);
    if (r <= c || c == n - 1) A[idx] = 0.0;
  }
}

}  // namespace

void tridiagonalize(Exec& ex, EigWork& w, int n, double* A) {
  if (n <= 0) return;
  TriParams p{};
  p.n = n; p.A = A; p.Wp = w.Wp; p.d = w.d; p.e = w.e; p.tau = w.tau; p.scal = w.scal;
  const int nrbt = ceil_div(n, TB);
  // partial buffers
  double* base = w.part;
  p.p_ss = base;                       base += ceil_div(n, RT) + 1;
  p.p_wv = base;                       base += ceil_div(n, RT) + 1;
  p.p_vw = base;                       base += (long long)nrbt * 2 * NBP;
  double* VW = base;                   base += (long long)n * 2 * NBP;
  double* WV = base;                   base += (long long)n * 2 * NBP;
  p.p_y = base;
  const int ncols = n - 1;  // columns with a reflector
  for (int k0 = 0; k0 < ncols; k0 += NBP) {
    const int nbp = std::min(NBP, ncols - k0);
    const int k1 = k0 + nbp;
    p.k0 = k0;
    for (int jj = 0; jj < nbp; ++jj) {
      const int i = k0 + jj;
      p.i = i; p.j = jj;
      // K1
      const int g1 = ceil_div(n - i, RT);
      p.n_ss = g1;
      {
        KScope ks(ex, MOLGW_K_TRIDIAG_PANEL, 4);
        k1_col_update<<<g1, RT, 0, ex.st>>>(p);
        const int g2 = std::max(1, ceil_div(n - i - 2, RT));
        k2_householder<<<g2, RT, 0, ex.st>>>(p);
        p.rb0 = (i + 1) / TB;
        p.nrb = nrbt - p.rb0;
        p.nchunk = ceil_div(p.nrb, TPC);
        k3_symv<<<p.nrb * p.nchunk, 256, 0, ex.st>>>(p);
        const int g4 = ceil_div(n - i - 1, RT);
        k4_wcol<<<g4, RT, 0, ex.st>>>(p);
        p.n_wv_prev = g4;
        p.n_wv = g4;
      }
    }
    // end of panel: last column's W correction, pack, trailing rank-2k update
    const int i = k1 - 1;
    p.i = i; p.j = nbp - 1;
    {
      KScope ks(ex, MOLGW_K_TRIDIAG_PANEL, 1);
      k5_finish<<<ceil_div(n - i - 1, RT), RT, 0, ex.st>>>(p, nbp, k1, VW, WV);
    }
    const int m = n - k1;
    if (m > 0) {
      GemmF64 g;
      g.M = m; g.N = m; g.K = 2 * nbp;
      g.A = VW; g.sa_m = 1; g.sa_k = m;
      g.B = WV; g.sb_k = m; g.sb_n = 1;     // B(k, j) = WV(j, k)
      g.C = A + k1 + (long long)k1 * n; g.sc_m = 1; g.sc_n = n;
      g.alpha = -1.0; g.beta = 1.0; g.lower_only = true;
      g.kclass = MOLGW_K_TRIDIAG_SYR2K;
      gemm_f64(ex, g);
    }
    p.j = 0;
  }
  {
    KScope ks(ex, MOLGW_K_TRIDIAG_PANEL, 2);
    k_last_diag<<<1, 32, 0, ex.st>>>(A, n, w.d);
    const long long total = (long long)n * n;
    k_clean<<<(int)std::min<long long>(ceil_div(total, 256), 152LL * 32), 256, 0, ex.st>>>(A, n);
  }
}

}  // namespace molgw
