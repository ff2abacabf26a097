// Float64 Householder tridiagonalisation of a symmetric matrix on the GPU.
//
// Blocked one-stage reduction in the manner of LAPACK's dsytrd/dlatrd (lower
// triangle), 64-column panels.  One persistent cooperative kernel runs a whole
// panel; for each column i of the panel it goes through three phases separated
// by grid-wide barriers:
//   P1  deferred updates of column i by the panel's earlier reflectors
//       (A(i:n,i) -= V W(i,:)^T + W V(i,:)^T), the previous column's rank-1 W
//       correction w += -tau/2 (w^T v) v, and partial sums of squares of the part
//       to annihilate;
//   P2  the reflector H_i = I - tau v v^T (beta = -sign(alpha) ||x||, LAPACK
//       dlarfg convention; every CTA derives it from the partial sums) and
//       y = A22 v over the not-yet-updated trailing matrix in 64x64 tiles (the
//       upper half through transposed lower tiles), v scaled on the fly, partial
//       sums per tile chunk (deterministic order), plus V^T v and W^T v;
//   P3  the W column w = tau (y - W V^T v - V W^T v), the scaled v written back,
//       partial sums of w^T v.
// After the panel the trailing matrix gets A -= V W^T + W V^T as one float64
// GEMM with K = 128 over the lower 64x64 tiles (diagonal tiles in full).
//
// Storage: A column-major, ld = n.  Every 64x64 diagonal tile is kept full
// (both halves); off-diagonal tiles only below the diagonal.  Upper tiles are
// never read.  Data written by other CTAs inside the kernel is read with
// ld.global.cg (L2), never from a possibly stale L1 line.
//
// On GB300 the FP64 pipe (~2 DFMA/clk/SM) rather than HBM bounds both the
// symmetric matrix-vector products (2 flops per 8-byte element) and the
// rank-2k updates, so every FP64 loop is spread over the whole GPU.
#include <algorithm>

#include "common.cuh"

namespace molgw {

namespace {

constexpr int NBP = 64;     // panel width
constexpr int TB = 64;      // tile size of the symmetric matrix-vector product
constexpr int RT = 256;     // threads per CTA; rows per work item of the panel-end packing
constexpr int RC = 64;      // rows per work item in P1/P3 (four threads per row)

struct GridBar {
  unsigned int count;
  unsigned int gen;
  int abort;
  int pad;
};

struct PanelParams {
  int n, k0, nbp, k1;
  double* A;
  double* Wp;               // n x NBP, column-major
  double* d; double* e; double* tau;
  double* scal;             // [0] alpha, [3] uncorrected W(i+1, j)
  double* p_ss;             // P1 partials
  double* p_vw;             // P2: per row block, 2*NBP values
  double* p_y;              // P2: per CTA, partial y over the row blocks its tile range covers
  double* p_wv;             // P3 partials
  double* VW; double* WV;   // packed [V W] and [W V] of rows >= k1
  GridBar* bar;
  int* status;
};

__device__ __forceinline__ double ldg_cg(const double* p) { return __ldcg(p); }

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a cooperative launch, with a bounded wait: after ~1 s
// without progress it latches MOLGW_E_TIMEOUT, raises the abort flag and
// returns false so that every CTA leaves the kernel.
__device__ bool grid_sync(GridBar* bar, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned int g = atomicAdd(&bar->gen, 0u);
    __threadfence();
    const unsigned int arrived = atomicAdd(&bar->count, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long spins = 0;
      while (ld_acquire(&bar->gen) == g) {
        if (*(volatile int*)&bar->abort != 0) { ok = 0; break; }
        if (++spins > (1LL << 24)) {
          set_status(status, MOLGW_E_TIMEOUT);
          atomicExch(&bar->abort, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

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

// Sum of `cnt` partials, the same value and order in every thread of every CTA.
__device__ double sum_partials(const double* p, int cnt, double* sh) {
  double v = 0.0;
  for (int k = threadIdx.x; k < cnt; k += blockDim.x) v += ldg_cg(p + k);
  double s = blk_reduce_sum(v, sh);
  __syncthreads();
  if (threadIdx.x == 0) sh[32] = s;
  __syncthreads();
  return sh[32];
}

struct Refl { double tau, beta, scale; };

__device__ Refl householder(const PanelParams& p, int i, double* sh) {
  const int n_ss = ceil_div_d(p.n - i, RC);
  const double sumsq = sum_partials(p.p_ss, n_ss, sh);
  const double alpha = ldg_cg(p.scal + 0);
  Refl h{0.0, alpha, 0.0};
  if (sumsq > 0.0) {
    const double nrm = sqrt(alpha * alpha + sumsq);
    h.beta = (alpha >= 0.0) ? -nrm : nrm;
    h.tau = (h.beta - alpha) / h.beta;
    h.scale = 1.0 / (alpha - h.beta);
  }
  return h;
}

// v_i[r] for r >= i+1 during P2/P3 (column i still holds the unscaled x).
__device__ __forceinline__ double vval(const PanelParams& p, int i, int r, double scale) {
  if (r == i + 1) return 1.0;
  return ldg_cg(p.A + r + (long long)i * p.n) * scale;
}

__global__ void __launch_bounds__(RT, 2) k_panel(PanelParams p) {
  __shared__ double sh[40];
  __shared__ double Wi[NBP], Vi[NBP], vtv[NBP], wtv[NBP];
  __shared__ double tile[TB * (TB + 1)];
  __shared__ double vJ[TB];
  __shared__ double red[4][TB];
  const int n = p.n, k0 = p.k0;
  const long long ld = n;
  double* A = p.A;
  const int t = threadIdx.x;
  const int nrbt = (n + TB - 1) / TB;

  for (int j = 0; j < p.nbp; ++j) {
    const int i = k0 + j;
    // ---------------- P1: column update ----------------
    double alpha_w = 0.0;
    if (j > 0) {
      const double s = sum_partials(p.p_wv, ceil_div_d(n - i, RC), sh);
      alpha_w = -0.5 * ldg_cg(p.tau + i - 1) * s;
    }
    for (int c = t; c < j; c += blockDim.x) {
      double w = ldg_cg(p.Wp + i + (long long)c * ld);
      if (c == j - 1) w = ldg_cg(p.scal + 3) + alpha_w;   // W(i, j-1) before its correction; v_{i-1}(i) = 1
      Wi[c] = w;
      Vi[c] = ldg_cg(A + i + (long long)(k0 + c) * ld);
    }
    __syncthreads();
    // 64 rows per chunk, four lanes per row share the loop over the panel's columns
    const int rl = t >> 2, q4 = t & 3;
    const int n1 = ceil_div_d(n - i, RC);
    for (int ch = blockIdx.x; ch < n1; ch += gridDim.x) {
      const int r = i + ch * RC + rl;
      double upd = 0.0, wcorr = 0.0;
      if (r < n) {
        if (j > 0) wcorr = ldg_cg(p.Wp + r + (long long)(j - 1) * ld) + alpha_w * ldg_cg(A + r + (long long)(i - 1) * ld);
#pragma unroll 4
        for (int c = q4; c < j; c += 4) {
          const double vr = ldg_cg(A + r + (long long)(k0 + c) * ld);
          const double wr = (c == j - 1) ? wcorr : ldg_cg(p.Wp + r + (long long)c * ld);
          upd += vr * Wi[c] + wr * Vi[c];
        }
      }
      upd += __shfl_xor_sync(0xffffffffu, upd, 1);
      upd += __shfl_xor_sync(0xffffffffu, upd, 2);
      double sq = 0.0;
      if (r < n && q4 == 0) {
        if (j > 0) p.Wp[r + (long long)(j - 1) * ld] = wcorr;
        const double a = ldg_cg(A + r + (long long)i * ld) - upd;
        A[r + (long long)i * ld] = a;
        if (r == i) p.d[i] = a;
        if (r == i + 1) p.scal[0] = a;
        if (r >= i + 2) sq = a * a;
      }
      const double s = blk_reduce_sum(sq, sh);
      if (t == 0) p.p_ss[ch] = s;
    }
    if (!grid_sync(p.bar, p.status)) return;

    // ---------------- P2: reflector and y = A22 v ----------------
    const Refl h = householder(p, i, sh);
    const int lo = i + 1;
    const int rb0 = lo / TB;
    const int nrb = nrbt - rb0;
    // the nrb x nrb tiles of A22, row-major, split into equal contiguous ranges
    const long long T = (long long)nrb * nrb;
    const long long f0 = (long long)blockIdx.x * T / gridDim.x;
    const long long f1 = (long long)(blockIdx.x + 1) * T / gridDim.x;
    if (f0 < f1) {
      const int rr = t % TB, cq = t / TB;
      const int q = t / TB, x = t % TB;
      double nxt[16];
      double vnxt = 0.0;
      auto load_tile = [&](long long f) {
        const int R = rb0 + (int)(f / nrb), J = rb0 + (int)(f % nrb);
        const int tr = (J >= R) ? J : R, tc = (J >= R) ? R : J;   // stored tile (tr >= tc)
        const int gr = tr * TB + rr;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int gc = tc * TB + cq + 4 * k;
          nxt[k] = (gr < n && gc < n) ? ldg_cg(A + gr + (long long)gc * ld) : 0.0;
        }
        if (t < TB) {
          const int r = J * TB + t;
          vnxt = (r >= lo && r < n) ? vval(p, i, r, h.scale) : 0.0;
        }
      };
      load_tile(f0);
      double acc = 0.0;
      bool dots = false;
      for (long long f = f0; f < f1; ++f) {
        const int R = rb0 + (int)(f / nrb), J = rb0 + (int)(f % nrb);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) tile[(cq + 4 * k) * (TB + 1) + rr] = nxt[k];
        if (t < TB) vJ[t] = vnxt;
        __syncthreads();
        if (f + 1 < f1) load_tile(f + 1);   // in flight while this tile is used
        double s = 0.0;
        if (J <= R) {
#pragma unroll
          for (int c = q * 16; c < q * 16 + 16; ++c) s += tile[c * (TB + 1) + x] * vJ[c];
        } else {
#pragma unroll
          for (int r = q * 16; r < q * 16 + 16; ++r) s += tile[x * (TB + 1) + r] * vJ[r];
        }
        acc += s;
        if (J == rb0) dots = true;
        if (f + 1 == f1 || (f + 1) % nrb == 0) {
          // end of this CTA's part of row block R: store its partial of y_R
          __syncthreads();
          red[q][x] = acc;
          if (dots && t < TB) {
            const int r = R * TB + t;
            vJ[t] = (r >= lo && r < n) ? vval(p, i, r, h.scale) : 0.0;
          }
          __syncthreads();
          if (t < TB) {
            const int r = R * TB + t;
            if (r < n) p.p_y[(long long)blockIdx.x * n + r] = red[0][t] + red[1][t] + red[2][t] + red[3][t];
          }
          if (dots) {
            // V^T v and W^T v over row block R: one warp per column, two rows per lane
            const int warp = t >> 5, lane = t & 31;
            for (int c = warp; c < 2 * j; c += RT / 32) {
              const int cc = (c < j) ? c : c - j;
              const double* col = (c < j) ? A + (long long)(k0 + cc) * ld : p.Wp + (long long)cc * ld;
              double d2 = 0.0;
#pragma unroll
              for (int h2 = 0; h2 < 2; ++h2) {
                const int rr2 = lane + 32 * h2;
                const int r = R * TB + rr2;
                if (r >= lo && r < n) d2 += ldg_cg(col + r) * vJ[rr2];
              }
              for (int o = 16; o > 0; o >>= 1) d2 += __shfl_xor_sync(0xffffffffu, d2, o);
              if (lane == 0) p.p_vw[(long long)(R - rb0) * (2 * NBP) + c] = d2;
            }
          }
          acc = 0.0;
          dots = false;
        }
      }
    }
    if (!grid_sync(p.bar, p.status)) return;

    // ---------------- P3: W column ----------------
    {
      // sum the per-row-block partials: one warp per column, lanes stride over blocks
      const int warp = t >> 5, lane = t & 31;
      for (int c = warp; c < 2 * j; c += RT / 32) {
        double s = 0.0;
        for (int R = lane; R < nrb; R += 32) s += ldg_cg(p.p_vw + (long long)R * (2 * NBP) + c);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) { if (c < j) vtv[c] = s; else wtv[c - j] = s; }
      }
    }
    __syncthreads();
    const int n3 = ceil_div_d(n - i - 1, RC);
    for (int ch = blockIdx.x; ch < n3; ch += gridDim.x) {
      const int r = lo + ch * RC + rl;
      double y = 0.0;
      if (r < n) {
        // partials of y_r from the CTAs whose tile ranges cover row block R
        const long long T = (long long)nrb * nrb;
        const long long fa = (long long)(r / TB - rb0) * nrb, fb = fa + nrb - 1;
        const int ca = (int)(((fa + 1) * gridDim.x - 1) / T), cb = (int)(((fb + 1) * gridDim.x - 1) / T);
        for (int c = ca + q4; c <= cb; c += 4) {
          // CTAs with an empty tile range wrote nothing
          if ((long long)c * T / gridDim.x == (long long)(c + 1) * T / gridDim.x) continue;
          y += ldg_cg(p.p_y + (long long)c * n + r);
        }
#pragma unroll 4
        for (int c = q4; c < j; c += 4) {
          y -= ldg_cg(p.Wp + r + (long long)c * ld) * vtv[c];
          y -= ldg_cg(A + r + (long long)(k0 + c) * ld) * wtv[c];
        }
      }
      y += __shfl_xor_sync(0xffffffffu, y, 1);
      y += __shfl_xor_sync(0xffffffffu, y, 2);
      double part = 0.0;
      if (r < n && q4 == 0) {
        const double w = h.tau * y;
        p.Wp[r + (long long)j * ld] = w;
        if (r == lo) p.scal[3] = w;
        const double v = vval(p, i, r, h.scale);
        part = w * v;
        if (r >= i + 2) A[r + (long long)i * ld] = v;
      }
      const double s = blk_reduce_sum(part, sh);
      if (t == 0) p.p_wv[ch] = s;
    }
    if (blockIdx.x == 0 && t == 0) {
      p.e[i] = h.beta;
      p.tau[i] = h.tau;
      A[(i + 1) + (long long)i * ld] = 1.0;
    }
    if (!grid_sync(p.bar, p.status)) return;
  }

  // ---------------- end of panel: last W correction and packing ----------------
  const int i = p.k1 - 1, j = p.nbp - 1;
  const double s = sum_partials(p.p_wv, ceil_div_d(n - i - 1, RC), sh);
  const double alpha_w = -0.5 * ldg_cg(p.tau + i) * s;
  const long long m = n - p.k1;
  const int n5 = ceil_div_d(n - i - 1, RT);
  for (int ch = blockIdx.x; ch < n5; ch += gridDim.x) {
    const int r = i + 1 + ch * RT + t;
    if (r >= n) continue;
    double* wc = p.Wp + r + (long long)j * ld;
    const double wnew = ldg_cg(wc) + alpha_w * ldg_cg(A + r + (long long)i * ld);
    *wc = wnew;
    if (r >= p.k1) {
      const long long rr = r - p.k1;
      for (int c = 0; c < p.nbp; ++c) {
        const double vv = ldg_cg(A + r + (long long)(k0 + c) * ld);
        const double ww = (c == j) ? wnew : ldg_cg(p.Wp + r + (long long)c * ld);
        p.VW[rr + (long long)c * m] = vv;
        p.VW[rr + (long long)(p.nbp + c) * m] = ww;
        p.WV[rr + (long long)c * m] = ww;
        p.WV[rr + (long long)(p.nbp + c) * m] = vv;
      }
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

int g_coop_blocks_per_sm = -1;   // the panel grid never exceeds kMaxPanelGrid (p_y has that many rows)
int g_num_sms = 0;

}  // namespace

void tridiagonalize(Exec& ex, EigWork& w, int n, double* A) {
  if (n <= 0) return;
  if (g_coop_blocks_per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_panel, RT, 0);
    g_coop_blocks_per_sm = std::max(1, std::min(occ, 2));
    g_coop_blocks_per_sm = std::min(g_coop_blocks_per_sm, kMaxPanelGrid / std::max(g_num_sms, 1));
  }
  PanelParams p{};
  p.n = n; p.A = A; p.Wp = w.Wp; p.d = w.d; p.e = w.e; p.tau = w.tau; p.scal = w.scal;
  p.status = ex.status;
  const int nrbt = ceil_div(n, TB);
  double* base = w.part;
  p.p_ss = base;   base += ceil_div(n, RC) + 1;
  p.p_wv = base;   base += ceil_div(n, RC) + 1;
  p.p_vw = base;   base += (long long)nrbt * 2 * NBP;
  p.VW = base;     base += (long long)n * 2 * NBP;
  p.WV = base;     base += (long long)n * 2 * NBP;
  p.bar = reinterpret_cast<GridBar*>(base);   base += 2;
  p.p_y = base;
  const int cap = g_num_sms * g_coop_blocks_per_sm;
  const int ncols = n - 1;
  for (int k0 = 0; k0 < ncols; k0 += NBP) {
    const int nbp = std::min(NBP, ncols - k0);
    const int k1 = k0 + nbp;
    p.k0 = k0; p.nbp = nbp; p.k1 = k1;
    const int nrb = nrbt - (k0 + 1) / TB;
    const long long tiles = (long long)nrb * nrb;
    const int grid = (int)std::max<long long>(1, std::min<long long>(cap, std::max<long long>(tiles, ceil_div(n - k0, RC))));
    {
      KScope ks(ex, MOLGW_K_TRIDIAG_PANEL, 1);
      cudaMemsetAsync(p.bar, 0, sizeof(GridBar), ex.st);
      void* args[] = {&p};
      cudaLaunchCooperativeKernel((const void*)k_panel, dim3(grid), dim3(RT), args, 0, ex.st);
    }
    const int m = n - k1;
    if (m > 0) {
      GemmF64 g;
      g.M = m; g.N = m; g.K = 2 * nbp;
      g.A = p.VW; g.sa_m = 1; g.sa_k = m;
      g.B = p.WV; g.sb_k = m; g.sb_n = 1;     // B(k, j) = WV(j, k)
      g.C = A + k1 + (long long)k1 * n; g.sc_m = 1; g.sc_n = n;
      g.alpha = -1.0; g.beta = 1.0; g.lower_only = true;
      g.kclass = MOLGW_K_TRIDIAG_SYR2K;
      gemm_f64(ex, g);
    }
  }
  {
    KScope ks(ex, MOLGW_K_TRIDIAG_PANEL, 2);
    k_last_diag<<<1, 32, 0, ex.st>>>(A, n, w.d);
    const long long total = (long long)n * n;
    k_clean<<<(int)std::min<long long>(ceil_div(total, 256), 152LL * 32), 256, 0, ex.st>>>(A, n);
  }
}

}  // namespace molgw
