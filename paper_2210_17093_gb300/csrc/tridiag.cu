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
#include "fx.cuh"

namespace molgw {

namespace {

constexpr int NBP = 64;     // panel width
constexpr int TB = 64;      // tile size of the symmetric matrix-vector product
constexpr int RT = 256;     // threads per CTA; rows per work item of the panel-end packing
constexpr int RC = 32;      // rows per work item in P1/P3 (eight threads per row)

struct GridBar {
  unsigned int count;
  unsigned int gen;
  int abort;
  int pad;
  unsigned int n0, n1;          // CTAs that were first on their SM, and the others
  unsigned int sm_slot[256];    // CTAs seen per SM id (mod 256)
};
static_assert(sizeof(GridBar) <= kGridBarDoubles * sizeof(double), "grid barrier block");

struct PanelParams {
  int n, k0, nbp, k1;
  double* A;
  double* Wp;               // n x NBP, column-major
  double* d; double* e; double* tau;
  double* scal;             // [0] alpha, [3] uncorrected W(i+1, j)
  double* p_ss;             // P1 partials
  double* p_vw;             // P1: per 32-row chunk, 2*NBP dot-product partials
  double* vwf;              // P2: the finished V^T v and W^T v (2*NBP)
  double* p_y;              // P2: per CTA, partial y over the row blocks its tile range covers
  double* p_t;              // P2: per lower tile, transposed partial of y (64 values)
  double* p_wv;             // P3 partials
  double* VW; double* WV;   // packed [V W] and [W V] of rows >= k1
  GridBar* bar;
  int* status;
  long long spin_limit;     // polls of a grid barrier before it gives up
};

__device__ __forceinline__ double ldg_cg(const double* p) { return __ldcg(p); }

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a cooperative launch.  Arrival is one fire-and-forget
// release increment of a counter that only grows during the launch (zeroed before
// it); barrier number e of the launch is passed when the counter reaches
// e * gridDim.x, seen with acquire loads.  The wait is bounded: after spin_limit
// polls (~1 s with the default) without progress it latches MOLGW_E_TIMEOUT, raises
// the abort flag and returns false so that every CTA leaves the kernel.  A CTA that
// arrives last passes; it leaves at its next barrier, where the abort flag stops
// its wait.
__device__ bool grid_sync(GridBar* bar, int* status, unsigned int& epoch, long long spin_limit) {
  __shared__ int ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned int target = epoch * gridDim.x;
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&bar->count) : "memory");
    long long spins = 0;
    while (ld_acquire(&bar->count) < target) {
      if (*(volatile int*)&bar->abort != 0) { ok = 0; break; }
      if (++spins > spin_limit) {
        set_status(status, MOLGW_E_TIMEOUT);
        atomicExch(&bar->abort, 1);
        ok = 0;
        break;
      }
      if (spins > 64) __nanosleep(32);
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

// Sum over a chunk's rows of values held by the lanes with (thread & 7) == 0 (four per
// warp, the rest zero): two shuffle steps per warp, eight warp sums in thread 0, where
// the result is valid.  Two __syncthreads, like blk_reduce_sum.
__device__ __forceinline__ double chunk_rows_sum(double v, double* sh) {
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;
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

struct Refl { double tau, beta, scale, alpha; };

__device__ Refl householder(const PanelParams& p, int i, double* sh) {
  const int n_ss = ceil_div_d(p.n - i, RC);
  const double sumsq = sum_partials(p.p_ss, n_ss, sh);
  const double alpha = ldg_cg(p.scal + 0);
  Refl h{0.0, alpha, 0.0, alpha};
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
  __shared__ double tile[TB * (TB + 1)];   // P1 scratch; P2 row-block sums [8][64]
  const int n = p.n, k0 = p.k0;
  const long long ld = n;
  double* A = p.A;
  const int t = threadIdx.x;
  const int nrbt = (n + TB - 1) / TB;
  unsigned int epoch = 0;                 // grid barriers passed in this launch
  // Order of the P1/P3 row chunks over the CTAs: the first CTA of every SM before any
  // second one, so that while the chunks are fewer than the SMs no SM runs two of
  // them (their float64 work would share one SM's float64 pipe).  Ranks come from
  // counters in the barrier block; the order is a permutation of 0..gridDim.x-1 and
  // takes effect after the first grid barrier, when the count of first CTAs is final.
  __shared__ int s_rank[3];
  if (t == 0) {
    unsigned int sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    const unsigned int slot = atomicAdd(&p.bar->sm_slot[sm & 255u], 1u);
    s_rank[0] = (slot == 0) ? 0 : 1;
    s_rank[1] = (int)atomicAdd((slot == 0) ? &p.bar->n0 : &p.bar->n1, 1u);
  }
  int L = blockIdx.x;

  for (int j = 0; j < p.nbp; ++j) {
    const int i = k0 + j;
    // ---------------- P1: column update ----------------
    // 32 rows per chunk, eight lanes per row share the loop over the panel's columns.
    // Besides the update, each chunk adds up V(r,:) a(r) and W(r,:) a(r) over its
    // rows r >= i+2 (a = the updated, still unscaled column): the dot products
    // V^T v and W^T v of P3 are these sums times the reflector's scale plus the
    // row i+1 terms (v(i+1) = 1).
    const int rl = t >> 3, q8 = t & 7;
    const int n1 = ceil_div_d(n - i, RC);
    double alpha_w = 0.0;
    if (j > 0) {
      const double s = sum_partials(p.p_wv, n1, sh);
      alpha_w = -0.5 * ldg_cg(p.tau + i - 1) * s;
    }
    if (t < j) {
      double w = ldg_cg(p.Wp + i + (long long)t * ld);
      if (t == j - 1) w = ldg_cg(p.scal + 3) + alpha_w;   // W(i, j-1) before its correction; v_{i-1}(i) = 1
      Wi[t] = w;
      Vi[t] = ldg_cg(A + i + (long long)(k0 + t) * ld);
    }
    __syncthreads();
    for (int ch = L; ch < n1; ch += gridDim.x) {
      const int r = i + ch * RC + rl;
      double upd = 0.0, wcorr = 0.0;
      double vs[NBP / 8], ws[NBP / 8];
      if (r < n && j > 0)
        wcorr = ldg_cg(p.Wp + r + (long long)(j - 1) * ld) + alpha_w * ldg_cg(A + r + (long long)(i - 1) * ld);
#pragma unroll
      for (int k = 0; k < NBP / 8; ++k) {
        const int c = q8 + 8 * k;
        vs[k] = 0.0;
        ws[k] = 0.0;
        if (r < n && c < j) {
          vs[k] = ldg_cg(A + r + (long long)(k0 + c) * ld);
          ws[k] = (c == j - 1) ? wcorr : ldg_cg(p.Wp + r + (long long)c * ld);
          upd += vs[k] * Wi[c] + ws[k] * Vi[c];
        }
      }
      upd += __shfl_xor_sync(0xffffffffu, upd, 1);
      upd += __shfl_xor_sync(0xffffffffu, upd, 2);
      upd += __shfl_xor_sync(0xffffffffu, upd, 4);
      double a = 0.0;
      if (r < n) a = ldg_cg(A + r + (long long)i * ld) - upd;
      double sq = 0.0;
      if (r < n && q8 == 0) {
        if (j > 0) p.Wp[r + (long long)(j - 1) * ld] = wcorr;
        A[r + (long long)i * ld] = a;
        if (r == i) p.d[i] = a;
        if (r == i + 1) p.scal[0] = a;
        if (r >= i + 2) sq = a * a;
      }
      // dot partials over the chunk's rows: the chunk's rows of V and W go to shared
      // memory (row stride 2 NBP + 1) with a(r) beside them, and two threads per column
      // sum sixteen rows each with fused multiply-adds (a third of the float64
      // instructions of a shuffle reduction, on a pipe that P1 otherwise saturates)
      const double aa = (r < n && r >= i + 2) ? a : 0.0;
      double* vw = tile;                         // [RC][2 NBP + 1]
      double* av = tile + RC * (2 * NBP + 1);    // [RC]
#pragma unroll
      for (int k = 0; k < NBP / 8; ++k) {
        vw[rl * (2 * NBP + 1) + q8 + 8 * k] = vs[k];
        vw[rl * (2 * NBP + 1) + NBP + q8 + 8 * k] = ws[k];
      }
      if (q8 == 0) av[rl] = aa;
      const double s = chunk_rows_sum(sq, sh);   // its __syncthreads publish vw and av
      if (t == 0) p.p_ss[ch] = s;
      {
        const int c = t >> 1, hf = t & 1;
        double d2 = 0.0;
        if (c < 2 * j) {
          const int col = (c < j) ? c : NBP + (c - j);
#pragma unroll
          for (int k = 0; k < RC / 2; ++k) {
            const int row = hf * (RC / 2) + k;
            d2 = fma(vw[row * (2 * NBP + 1) + col], av[row], d2);
          }
        }
        d2 += __shfl_xor_sync(0xffffffffu, d2, 1);
        if (c < 2 * j && hf == 0) p.p_vw[(long long)ch * (2 * NBP) + c] = d2;
      }
      __syncthreads();
    }
    if (!grid_sync(p.bar, p.status, epoch, p.spin_limit)) return;
    if (j == 0) {
      if (t == 0) s_rank[2] = (s_rank[0] == 0) ? s_rank[1] : (int)ld_acquire(&p.bar->n0) + s_rank[1];
      __syncthreads();
      L = s_rank[2];
    }

    // ---------------- P2: reflector and y = A22 x ----------------
    // The symmetric product runs on the unscaled column x (rows >= i+1 of column i as
    // P1 left it, x_(i+1) = alpha): v = scale x + (1 - scale alpha) e_(i+1), so P3 forms
    // A22 v = scale (A22 x) + (1 - scale alpha) A22 e_(i+1) from the partials written here.
    const int lo = i + 1;
    const int rb0 = lo / TB;
    const int nrb = nrbt - rb0;
    // The stored (lower and diagonal) tiles of A22 in row-major order (R, J <= R),
    // split into equal contiguous ranges.  Each tile is read once into registers and
    // used twice: y_R += A_RJ x_J (per thread along its rows, summed over the CTA at
    // the end of its part of row block R, stored per CTA and row block) and, below the
    // diagonal, y_J += A_RJ^T x_R (summed over the tile's rows by shuffles, stored per
    // tile).  Thread (warp w, lane l) holds rows (l & 15) + 16 k and columns
    // 8 w + 4 (l >> 4) + c of the tile (k, c < 4): every load instruction reads 128
    // contiguous bytes per half-warp, and no shared memory or barrier is used per tile.
    const long long T = (long long)nrb * (nrb + 1) / 2;
    const long long f0 = (long long)blockIdx.x * T / gridDim.x;
    const long long f1 = (long long)(blockIdx.x + 1) * T / gridDim.x;
    const int wq = t >> 5, lane = t & 31, rq = lane & 15;
    const int cq0 = 8 * wq + 4 * (lane >> 4);
    double nxt[16];                        // [4 c + k]
    // (R, J) of the first tile of the range: R - rb0 = the largest a with a(a+1)/2 <= f0
    // (integer search; later tiles advance J, then R).  Its elements are loaded before
    // the reflector's norm is summed.
    int R0 = rb0, J0 = rb0;
    auto load_tile = [&](int R, int J) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int gc = J * TB + cq0 + c;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int gr = R * TB + rq + 16 * k;
          nxt[4 * c + k] = (gr < n && gc < n) ? __ldca(A + gr + (long long)gc * ld) : 0.0;
        }
      }
    };
    if (f0 < f1) {
      long long a = 0;
      while ((a + 1) * (a + 2) / 2 <= f0) ++a;
      R0 = rb0 + (int)a;
      J0 = rb0 + (int)(f0 - a * (a + 1) / 2);
      load_tile(R0, J0);
    }
    const Refl h = householder(p, i, sh);
    {
      // V^T v = V(i+1,:) + scale * (sum over the P1 chunks), the same for W^T v:
      // the first CTAs finish these 2j sums (one warp per value) for P3
      const int c = blockIdx.x * (RT / 32) + wq;
      if (c < 2 * j) {
        double s2 = 0.0;
        for (int ch = lane; ch < n1; ch += 32) s2 += ldg_cg(p.p_vw + (long long)ch * (2 * NBP) + c);
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) {
          const double row1 = (c < j) ? ldg_cg(A + lo + (long long)(k0 + c) * ld) : ldg_cg(p.Wp + lo + (long long)(c - j) * ld);
          p.vwf[c] = row1 + h.scale * s2;
        }
      }
    }
    if (f0 < f1) {
      // x entries of rows >= lo (written by P1 of this column: read through L2)
      auto xval = [&](int r) { return (r >= lo && r < n) ? ldg_cg(A + r + (long long)i * ld) : 0.0; };
      double acc[4] = {0.0, 0.0, 0.0, 0.0};   // y_R partials of the thread's rows
      double xr[4];
      int R = R0, J = J0;
#pragma unroll
      for (int k = 0; k < 4; ++k) xr[k] = xval(R * TB + rq + 16 * k);
      for (long long f = f0; f < f1; ++f) {
        int Rn = R, Jn = J + 1;             // next tile
        if (Jn > Rn) { ++Rn; Jn = rb0; }
        double cur[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) cur[e] = nxt[e];
        double xc[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) xc[c] = xval(J * TB + cq0 + c);
        if (f + 1 < f1) load_tile(Rn, Jn);   // in flight while this tile is used
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[k] = fma(cur[4 * c + k], xc[c], acc[k]);
        if (J < R) {
          double q[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            q[c] = cur[4 * c] * xr[0];
#pragma unroll
            for (int k = 1; k < 4; ++k) q[c] = fma(cur[4 * c + k], xr[k], q[c]);
          }
          // sum over the 16 lanes of the half-warp (the tile's 64 rows), scattering the
          // four columns: lane bits 3 and 2 select the column each lane keeps
          const bool b3 = (rq & 8) != 0, b2 = (rq & 4) != 0;
          const double k0v = b3 ? q[2] : q[0], k1v = b3 ? q[3] : q[1];
          const double s0v = b3 ? q[0] : q[2], s1v = b3 ? q[1] : q[3];
          const double h0 = k0v + __shfl_xor_sync(0xffffffffu, s0v, 8);
          const double h1 = k1v + __shfl_xor_sync(0xffffffffu, s1v, 8);
          double v = (b2 ? h1 : h0) + __shfl_xor_sync(0xffffffffu, b2 ? h0 : h1, 4);
          v += __shfl_xor_sync(0xffffffffu, v, 2);
          v += __shfl_xor_sync(0xffffffffu, v, 1);
          if ((rq & 3) == 0) {
            const long long ft = (long long)(R - rb0) * (R - rb0 + 1) / 2 + (J - rb0);
            p.p_t[ft * TB + cq0 + 2 * (b3 ? 1 : 0) + (b2 ? 1 : 0)] = v;
          }
        }
        if (f + 1 == f1 || J == R) {
          // end of this CTA's part of row block R: the rows' sums over the 16 threads that
          // hold them (the two half-warps, then the eight warps through shared memory)
          double* red = tile;               // [8][64]
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], 16);
          __syncthreads();
          if (lane < 16) {
#pragma unroll
            for (int k = 0; k < 4; ++k) red[wq * TB + rq + 16 * k] = acc[k];
          }
          __syncthreads();
          if (t < TB) {
            double y = red[t];
#pragma unroll
            for (int w2 = 1; w2 < RT / 32; ++w2) y += red[w2 * TB + t];
            const int r = R * TB + t;
            if (r < n) p.p_y[(long long)blockIdx.x * n + r] = y;
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[k] = 0.0;
          if (f + 1 < f1 && Rn != R) {
#pragma unroll
            for (int k = 0; k < 4; ++k) xr[k] = xval(Rn * TB + rq + 16 * k);
          }
        }
        R = Rn;
        J = Jn;
      }
    }
    if (!grid_sync(p.bar, p.status, epoch, p.spin_limit)) return;

    // ---------------- P3: W column ----------------
    const int n3 = ceil_div_d(n - i - 1, RC);
    for (int c = t; c < 2 * j; c += blockDim.x) {
      const double v = ldg_cg(p.vwf + c);
      if (c < j) vtv[c] = v; else wtv[c - j] = v;
    }
    __syncthreads();
    for (int ch = L; ch < n3; ch += gridDim.x) {
      const int r = lo + ch * RC + rl;
      double y = 0.0;
      if (r < n) {
        // (A22 x)_r = (direct partials of the CTAs whose ranges cover row block R)
        //           + (transposed partials of the tiles (R', R) below it);
        // y_r = scale (A22 x)_r + (1 - scale alpha) A(r, i+1) - W(r,:) V^T v - V(r,:) W^T v
        const int Rr = r / TB, a = Rr - rb0;
        const long long T = (long long)nrb * (nrb + 1) / 2;
        const long long fa = (long long)a * (a + 1) / 2, fb = fa + a;
        const int ca = (int)(((fa + 1) * gridDim.x - 1) / T), cb = (int)(((fb + 1) * gridDim.x - 1) / T);
        double yx = 0.0;
        for (int c = ca + q8; c <= cb; c += 8) {
          // CTAs with an empty tile range wrote nothing
          if ((long long)c * T / gridDim.x == (long long)(c + 1) * T / gridDim.x) continue;
          yx += ldg_cg(p.p_y + (long long)c * n + r);
        }
#pragma unroll 8
        for (int R2 = Rr + 1 + q8; R2 < nrbt; R2 += 8) {
          const long long ft = (long long)(R2 - rb0) * (R2 - rb0 + 1) / 2 + a;
          yx += ldg_cg(p.p_t + ft * TB + (r - Rr * TB));
        }
        if (q8 == 0) y = (1.0 - h.scale * h.alpha) * ldg_cg(A + r + (long long)(i + 1) * ld);
#pragma unroll 4
        for (int c = q8; c < j; c += 8) {
          y -= ldg_cg(p.Wp + r + (long long)c * ld) * vtv[c];
          y -= ldg_cg(A + r + (long long)(k0 + c) * ld) * wtv[c];
        }
        y = fma(h.scale, yx, y);
      }
      y += __shfl_xor_sync(0xffffffffu, y, 1);
      y += __shfl_xor_sync(0xffffffffu, y, 2);
      y += __shfl_xor_sync(0xffffffffu, y, 4);
      double part = 0.0;
      if (r < n && q8 == 0) {
        const double w = h.tau * y;
        p.Wp[r + (long long)j * ld] = w;
        if (r == lo) p.scal[3] = w;
        const double v = vval(p, i, r, h.scale);
        part = w * v;
        if (r >= i + 2) A[r + (long long)i * ld] = v;
      }
      const double s = chunk_rows_sum(part, sh);
      if (t == 0) p.p_wv[ch] = s;
    }
    if (blockIdx.x == 0 && t == 0) {
      p.e[i] = h.beta;
      p.tau[i] = h.tau;
      A[(i + 1) + (long long)i * ld] = 1.0;
    }
    if (!grid_sync(p.bar, p.status, epoch, p.spin_limit)) return;
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

int tridiag_coop_capacity() {
  if (g_coop_blocks_per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_panel, RT, 0);
    g_coop_blocks_per_sm = std::max(1, std::min(occ, 2));
    g_coop_blocks_per_sm = std::min(g_coop_blocks_per_sm, kMaxPanelGrid / std::max(g_num_sms, 1));
  }
  return g_num_sms * g_coop_blocks_per_sm;
}

void tridiagonalize(Exec& ex, EigWork& w, int n, double* A) {
  if (n <= 0) return;
  tridiag_coop_capacity();
  PanelParams p{};
  p.n = n; p.A = A; p.Wp = w.Wp; p.d = w.d; p.e = w.e; p.tau = w.tau; p.scal = w.scal;
  p.status = ex.status;
  p.spin_limit = ex.grid_spins;
  const int nrbt = ceil_div(n, TB);
  double* base = w.part;
  p.p_ss = base;   base += ceil_div(n, RC) + 1;
  p.p_wv = base;   base += ceil_div(n, RC) + 1;
  p.p_vw = base;   base += ((long long)ceil_div(n, RC) + 1) * 2 * NBP;
  p.vwf = base;    base += 2 * NBP;
  p.VW = base;     base += (long long)n * 2 * NBP;
  p.WV = base;     base += (long long)n * 2 * NBP;
  p.bar = reinterpret_cast<GridBar*>(base);   base += kGridBarDoubles;
  p.p_t = base;    base += (long long)nrbt * (nrbt + 1) / 2 * TB;
  p.p_y = base;
  // Concurrent lanes each take a share of the co-resident CTAs, so that the
  // persistent panels of all lanes fit on the device at the same time.
  int cap = g_num_sms * g_coop_blocks_per_sm;
  if (ex.coop_cap > 0) cap = std::max(2 * NBP / (RT / 32), std::min(cap, ex.coop_cap));
  const int ncols = n - 1;
  for (int k0 = 0; k0 < ncols; k0 += NBP) {
    const int nbp = std::min(NBP, ncols - k0);
    const int k1 = k0 + nbp;
    p.k0 = k0; p.nbp = nbp; p.k1 = k1;
    const int nrb = nrbt - (k0 + 1) / TB;
    const long long tiles = (long long)nrb * (nrb + 1) / 2;
    const int grid = (int)std::max<long long>(2 * NBP / (RT / 32),
                                               std::min<long long>(cap, std::max<long long>(tiles, ceil_div(n - k0, RC))));
    {
      KScope ks(ex, MOLGW_K_TRIDIAG_PANEL, 1);
      cudaMemsetAsync(p.bar, 0, sizeof(GridBar), ex.st);
      void* args[] = {&p};
      cudaLaunchCooperativeKernel((const void*)k_panel, dim3(grid), dim3(RT), args, 0, ex.st);
    }
    const int m = n - k1;
    if (m > 0 && w.fx && m <= w.fx_rows && m >= 128) {
      // A22 -= [V W] [W V]^T on the tensor cores: 7-digit fixed point, exact sums
      const int kk = (int)fx_pad(2 * nbp);
      FxMat a = fx_mat_carve(w.fx, m, 128, 7);
      FxMat b = fx_mat_carve((char*)w.fx + fx_mat_bytes(w.fx_rows, 128, 7), m, 128, 7);
      fx_split(ex, p.VW, m, 2 * nbp, 1, m, nullptr, a, MOLGW_K_TRIDIAG_SYR2K);
      fx_split(ex, p.WV, m, 2 * nbp, 1, m, nullptr, b, MOLGW_K_TRIDIAG_SYR2K);
      FxGemm g;
      g.M = m; g.N = m; g.K = kk;
      g.A = a; g.B = b;
      g.out = A + k1 + (long long)k1 * n;
      g.out_ld = n;
      g.col_major = true;
      g.accumulate = true;
      g.alpha = -1.0;
      g.lower_only = true;
      g.kclass = MOLGW_K_TRIDIAG_SYR2K;
      fx_gemm(ex, g);
    } else if (m > 0) {
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
