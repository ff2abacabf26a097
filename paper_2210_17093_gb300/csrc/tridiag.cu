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
  // tensor-core mat-vec (k_panel<true>): tile images and scales of the panel's trailing
  // region (tile index relative to block k0 / 64), P1's column-maximum partials
  const uint8_t* sv_img;
  const double* sv_scl;
  double* sv_mx;
  // integer mat-vec (k_panel<kPanelInt>): the trailing region's lower tiles as 53-bit
  // fixed point (tile index relative to block k0 / 64) and each row block's exponent
  const long long* ix_img;
  const int* ix_texp;       // e_T per tile (as ix_img)
  const unsigned long long* ix_gmax;   // bit pattern of the largest |a| of all tiles
};

__device__ __forceinline__ double ldg_cg(const double* p) { return __ldcg(p); }

// (R, J) of lower tile f counted row by row from block rbp: R - rbp = the largest a with
// a(a+1)/2 <= f (a float32 square root as the estimate, exact integer fix-ups)
__device__ __forceinline__ void tile_of(long long f, int rbp, int& R, int& J) {
  long long a = (long long)((sqrtf(8.0f * (float)f + 1.0f) - 1.0f) * 0.5f);
  if (a < 0) a = 0;
  while (a > 0 && a * (a + 1) / 2 > f) --a;
  while ((a + 1) * (a + 2) / 2 <= f) ++a;
  R = rbp + (int)a;
  J = rbp + (int)(f - a * (a + 1) / 2);
}

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
__device__ bool grid_sync(GridBar* bar, int* status, unsigned int& epoch, long long spin_limit, int leader = 0) {
  __shared__ int ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == leader) {
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

// Reductions of the panel kernel.  On GB300 a float64 warp instruction occupies the SM's
// float64 pipe for the same ~19 cycles however many of its lanes are active, so a sum
// over the CTA is formed by one warp: every thread's value goes to shared memory
// (sh[kShBuf + t], RT doubles), warp 0 adds eight of them per lane and finishes with five
// shuffle steps.  sh[0..39] hold scalars; every helper starts with a __syncthreads (which
// also publishes the caller's earlier shared-memory writes) and returns after another.
constexpr int kShBuf = 40;

// Sum of the values v of all threads in a fixed order; valid in every thread.
__device__ double cta_sum(double v, double* sh) {
  const int t = threadIdx.x;
  __syncthreads();
  sh[kShBuf + t] = v;
  __syncthreads();
  if (t < 32) {
    double s = sh[kShBuf + t];
#pragma unroll
    for (int k = 1; k < RT / 32; ++k) s += sh[kShBuf + t + 32 * k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (t == 0) sh[32] = s;
  }
  __syncthreads();
  return sh[32];
}

// Sum over a chunk's rows of values held by the lanes with (thread & 7) == 0 (the rest
// zero): the 32 row values go to shared memory and warp 0 adds them.  Valid in thread 0;
// its first __syncthreads publishes the caller's shared-memory writes.
__device__ __forceinline__ double chunk_rows_sum(double v, double* sh) {
  const int t = threadIdx.x;
  __syncthreads();
  if ((t & 7) == 0) sh[kShBuf + (t >> 3)] = v;
  __syncthreads();
  double s = 0.0;
  if (t < 32) {
    s = sh[kShBuf + t];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}

// Sum of `cnt` partials, the same value and order in every thread of every CTA.
__device__ double sum_partials(const double* p, int cnt, double* sh, double v0) {
  const int t = threadIdx.x;
  double v = v0;
  for (int k = t + RT; k < cnt; k += RT) v += ldg_cg(p + k);
  return cta_sum(v, sh);
}
__device__ double sum_partials(const double* p, int cnt, double* sh) {
  return sum_partials(p, cnt, sh, (threadIdx.x < cnt) ? ldg_cg(p + threadIdx.x) : 0.0);
}

struct Refl { double tau, beta, scale, alpha; };

// Sum of `cnt` partials ps[] and the largest of the non-negative pm[] (compared as
// 64-bit integers: the bit patterns of non-negative doubles are ordered like their
// values), both the same in every thread of every CTA.
__device__ double sum_max_partials(const double* ps, const double* pm, int cnt, double* sh, double& mx, double v0,
                                  long long m0) {
  const int t = threadIdx.x;
  double v = v0;
  long long m = m0;
  for (int k = t + RT; k < cnt; k += RT) {
    v += ldg_cg(ps + k);
    m = max(m, __double_as_longlong(ldg_cg(pm + k)));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  __syncthreads();
  if ((t & 31) == 0) reinterpret_cast<long long*>(sh)[16 + (t >> 5)] = m;
  const double s = cta_sum(v, sh);   // its __syncthreads publish the warp maxima
  long long mm = 0;
#pragma unroll
  for (int w = 0; w < RT / 32; ++w) mm = max(mm, reinterpret_cast<long long*>(sh)[16 + w]);
  mx = __longlong_as_double(mm);
  return s;
}

// The reflector of column i from P1's partial sums of squares (LAPACK dlarfg
// convention), computed by thread 0 and shared; with xmax, also the largest |x_r| from
// P1's chunk maxima (the fixed-point mat-vecs' scale of x).  v0 and m0 are this thread's
// first partials (entry threadIdx.x, or 0), loaded by the caller ahead of other traffic.
__device__ Refl householder(const PanelParams& p, int n_ss, double* sh, double v0, long long m0,
                            double* xmax = nullptr) {
  const double sumsq = xmax ? sum_max_partials(p.p_ss, p.sv_mx, n_ss, sh, *xmax, v0, m0)
                            : sum_partials(p.p_ss, n_ss, sh, v0);
  if (threadIdx.x == 0) {
    const double alpha = ldg_cg(p.scal + 0);
    Refl h{0.0, alpha, 0.0, alpha};
    if (sumsq > 0.0) {
      const double nrm = sqrt(alpha * alpha + sumsq);
      h.beta = (alpha >= 0.0) ? -nrm : nrm;
      h.tau = (h.beta - alpha) / h.beta;
      h.scale = 1.0 / (alpha - h.beta);
    }
    sh[34] = h.tau;
    sh[35] = h.beta;
    sh[36] = h.scale;
    sh[37] = h.alpha;
  }
  __syncthreads();
  return Refl{sh[34], sh[35], sh[36], sh[37]};
}

// v_i[r] for r >= i+1 during P2/P3 (column i still holds the unscaled x).
__device__ __forceinline__ double vval(const PanelParams& p, int i, int r, double scale) {
  if (r == i + 1) return 1.0;
  return ldg_cg(p.A + r + (long long)i * p.n) * scale;
}

// ---------------------------------------------------------------------------
// Integer symmetric mat-vec (k_panel<kPanelInt>, MOLGW_FLAG_EIG_TC).  Before a panel,
// every stored 64 x 64 tile T of the trailing matrix is written as 53-bit fixed point on
// its own grid: a = m 2^(e_T - 53), m = rint(a 2^(53 - e_T)) with max |a| over the tile
// below 2^(e_T), so |m| <= 2^53, stored as m = h 2^27 + l (|h| <= 2^26,
// -2^26 <= l < 2^26) in one 64-bit word (l low, h high), tile-local column-major
// (element (r, c) at c * 64 + r).  In P2 x is put on one grid too, x = m_x 2^(e_x - 53)
// (|x| < 2^(e_x)), split the same way, and every product is
//   a x = [h h_x 2^54 + (h l_x + l h_x) 2^27 + l l_x] 2^(e_T + e_x - 106),
// formed with 32 x 32 -> 64-bit integer multiply-adds, exact; the last term (below
// 2^-54 of the grid's unit, of either sign) is left out and the middle sum is rounded to
// a multiple of 2^27 once per thread's four elements of a row (rounded, not floored: a
// floor would bias every row sum by n/8 units), giving 64-bit sums in units of
// 2^(e_T + e_x - 52).  Those
// are moved to the common grid 2^(e_g - 56 + e_x - 52) (e_g: the largest tile exponent)
// by left shifts of at most 56 places, exact, and added in 128 bits (below 2^125 for
// up to 1024 tiles per row), then rounded to float64 once per row; tiles more than
// 2^56 below the largest are shifted right instead.  Accuracy: every value is
// represented to 2^-54 of its tile's largest and x to 2^-54 of its largest, i.e.
// float64 accuracy in the normwise sense, not float64 arithmetic.  Throughput: a GB300 SM issues ~62 such multiply-adds per clock against
// 1.7 float64 FMAs, so the mat-vec is bound by reading the image (8 bytes per element,
// as float64) instead of the float64 pipe.
constexpr int kPanelF64 = 0, kPanelTc = 1, kPanelInt = 2;
constexpr long long kIxTileBytes = 64LL * 64 * 8;
static_assert(kIxTileBytes <= kSvTileBytes, "the integer image fits where the tensor-core image goes");

// rint(x 2^p) from the bit pattern (integer instructions only; the scaling by a power
// of two is exact, the rounding to nearest with ties to even); |x| 2^p must stay below
// 2^62.  Zero and subnormal x give 0.
__device__ __forceinline__ long long fixed_round(double x, int p) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex == 0) return 0;
  const unsigned long long m = (bits & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  const int sh = ex - 1075 + p;                          // x = m 2^(ex - 1075)
  unsigned long long t;
  if (sh >= 0) {
    t = m << sh;
  } else if (sh > -64) {
    const int r = -sh;
    t = (r < 64) ? (m >> r) : 0ULL;
    const unsigned long long rem = m & ((1ULL << r) - 1), half = 1ULL << (r - 1);
    if (rem > half || (rem == half && (t & 1ULL))) ++t;
  } else {
    t = 0;
  }
  return (bits >> 63) ? -(long long)t : (long long)t;
}
// c + a b with a 32 x 32 -> 64-bit product (one widening integer multiply-add)
__device__ __forceinline__ long long mad_wide(int a, int b, long long c) {
  long long d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}
// m = h 2^27 + l with l in [-2^26, 2^26)
__device__ __forceinline__ void split27(long long m, int& h, int& l) {
  h = (int)((m + (1LL << 26)) >> 27);
  l = (int)(m - ((long long)h << 27));
}
// 2^e as a float64 (e within the normal range; others through ldexp)
__device__ __forceinline__ double pow2i(int e) {
  return (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52) : ldexp(1.0, e);
}
// the exponent e with |v| < 2^e for the largest |v| of a group (0 for an all-zero group)
__device__ __forceinline__ int grid_exp(double vmax) {
  int e = 0;
  if (vmax > 0.0) frexp(vmax, &e);
  return e;
}

// The integer image of every stored tile (R, J), rbp <= J <= R, one CTA per tile: the
// tile's largest |a| (a maximum of bit patterns, ordered like the values: integer
// instructions), its exponent texp[f] = e_T, the elements on that grid, and an atomic
// maximum of the bit patterns into *gmax (zero before the launch).
__global__ void __launch_bounds__(256) k_ix_image(const double* __restrict__ A, int n, int rbp, long long* img,
                                                  int* texp, unsigned long long* gmax) {
  __shared__ unsigned long long red[8];
  int R, J;
  tile_of(blockIdx.x, rbp, R, J);
  const int t = threadIdx.x, r = t & 63, c0 = t >> 6;
  const int gr = R * TB + r;
  double v[16];
  unsigned long long mx = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int gc = J * TB + c0 + 4 * k;
    v[k] = (gr < n && gc < n) ? A[gr + (long long)gc * n] : 0.0;
    mx = max(mx, (unsigned long long)__double_as_longlong(v[k]) & 0x7FFFFFFFFFFFFFFFULL);
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((t & 31) == 0) red[t >> 5] = mx;
  __syncthreads();
  unsigned long long m = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = max(m, red[w]);
  const int e = grid_exp(__longlong_as_double((long long)m));
  long long* base = img + (long long)blockIdx.x * (TB * TB);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    int h, l;
    split27(fixed_round(v[k], 53 - e), h, l);
    base[(c0 + 4 * k) * TB + r] = (long long)(((unsigned long long)(unsigned int)h << 32) | (unsigned int)l);
  }
  if (t == 0) {
    texp[blockIdx.x] = e;
    atomicMax(gmax, m);
  }
}

// acc += v 2^s for s in [-63, 63] (a right shift, floor, for s < 0): the 128-bit shifted
// value from two 64-bit shifts, no branch on the shift count
__device__ __forceinline__ void add_shifted(__int128& acc, long long v, int s) {
  if (s >= 0) {
    const unsigned long long lo = (unsigned long long)v << s;
    const long long hi = (v >> 1) >> (63 - s);
    acc += ((__int128)hi << 64) | (__int128)lo;
  } else {
    acc += (__int128)(v >> min(-s, 63));
  }
}

// 128-bit integer to float64 (two roundings, relative error below 2^-52)
__device__ __forceinline__ double i128_to_f64(__int128 v) {
  const long long hi = (long long)(v >> 64);
  const unsigned long long lo = (unsigned long long)v;
  return fma((double)hi, 0x1p64, (double)lo);
}

// ---------------------------------------------------------------------------
// Tensor-core symmetric mat-vec (MOLGW_FLAG_EIG_TC).  Before a panel, every stored
// 64 x 64 tile of the trailing matrix is written as a 7-digit fixed-point image
// (fx.cuh: x ~ u sum_d s_d 2^(-8d), one power-of-two scale u per tile): digit plane d
// holds row c (tile column) = the 64 tile rows of column c, 128 bytes with the 128-byte
// swizzle, i.e. the shared-memory image a K-major operand indexed (column, row) and an
// MN-major operand indexed (row, column) both read.  In P2 the panel kernel copies
// tile images with the bulk-copy engine, writes the 7 digits of the two 64-blocks of x
// it needs (one scale per column: its maximum), and per tile issues, for each pair of
// digit planes (2g, 2g+1) of the tile and K step, M=128 N=8 K=16 MMAs: A_RJ x_J with the
// two planes as an MN-major A operand (64-element atoms 8 KB apart) and (below the
// diagonal) A_RJ^T x_R as a K-major one (the planes' rows contiguous), the 7 digits of x
// as the 8 columns of B.  (Each tcgen05.mma costs the same ~65 SM cycles whatever its
// shape at these sizes, so two planes per instruction halve the mat-vec's issue time.)
// TMEM lanes 0-63 then hold digit 2g's sums, lanes 64-127 digit 2g+1's: every column one
// digit pair's sum over 64 elements, an integer below 2^21, exact in float32.  The
// epilogue adds the pairs with i + j <= 6 into levels exactly (odd-digit warps hand their
// partial levels to the even-digit warps through shared memory), combines the levels in
// 64-bit integers (as the fixed-point GEMM does) and rounds once to float64.
// The arithmetic is float64-accurate in the normwise sense (values represented to
// 2^-54 of their tile's or column's largest), not float64 arithmetic.
constexpr int SV_PLANE = TB * TB * 2;                 // 8 KB: one digit plane of a tile image
constexpr int SV_TILE = 7 * SV_PLANE;                 // 57,344 B
constexpr int SV_XIMG = 8 * 128;                      // a 64-block of x: 7 digit rows + a zero row
constexpr int SV_STAGES = 3;
constexpr int SV_STAGE = SV_TILE + 2 * SV_XIMG;
// 1024 for the stage alignment, 8 KB so that the last digit pair's second half (a plane
// past the 7th, read and discarded) stays inside the allocation
constexpr int SV_SMEM = SV_STAGES * SV_STAGE + 1024 + SV_PLANE;
constexpr int SV_TMEM = 128;                          // 2 buffers x (32 + 32) columns
constexpr long long SV_SPIN = 1LL << 26;
static_assert(SV_TILE == kSvTileBytes, "tile image size");
static_assert(SV_STAGE % 1024 == 0, "stages stay 1024-byte aligned");

// byte offset of 16-bit element e of row `row` of a 128-byte-row image, 128-byte swizzle
__device__ __forceinline__ int sv_sw(int row, int e) {
  return row * 128 + ((((e * 2) >> 4) ^ (row & 7)) << 4) + ((e * 2) & 15);
}
__device__ __forceinline__ uint32_t sv_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// matrix descriptor: 128-byte swizzle, leading / stride byte offsets
__device__ __forceinline__ uint64_t sv_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((sv_u32(p) & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__device__ __forceinline__ void sv_mbar_init(uint64_t* b, uint32_t cnt) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sv_u32(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ bool sv_mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t done;
  asm volatile("{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}"
               : "=r"(done) : "r"(sv_u32(b)), "r"(parity) : "memory");
  return done != 0;
}
// bounded wait; gives up early when *abort is raised (checked every 256 polls)
__device__ __forceinline__ bool sv_wait(uint64_t* b, uint32_t parity, volatile int* abort) {
  for (long long it = 0; it < SV_SPIN; ++it) {
    if (sv_mbar_try(b, parity)) return true;
    if ((it & 255) == 255 && *abort) return false;
  }
  return false;
}
__device__ __forceinline__ void sv_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
               "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void sv_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sv_u32(b)) : "memory");
}
__device__ __forceinline__ void sv_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
// The 7 digits of x / u (u = 2^(e-7), |x| < 2^e) as fx_digits<7>(x, 2^48 / u) writes them,
// with integer instructions only: T = rint(x 2^(55-e)) from the bit pattern (the scaling
// by a power of two is exact, the rounding is to nearest, ties to even), then the
// balanced base-256 digits.
__device__ __forceinline__ void sv_digits7(double x, int e, __nv_bfloat16* out) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long T = 0;
  if (ex != 0) {                                        // zero and subnormals (far below u) give 0
    const unsigned long long m = (bits & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
    const int sh = (ex - 1023) - 52 + 55 - e;          // value = m 2^(ex-1075), times 2^(55-e)
    unsigned long long t;
    if (sh >= 0) {
      t = m << sh;                                      // sh <= 2 since |x| < 2^e
    } else if (sh > -64) {
      const int r = -sh;
      t = m >> r;
      const unsigned long long rem = m & ((1ULL << r) - 1), half = 1ULL << (r - 1);
      if (rem > half || (rem == half && (t & 1ULL))) ++t;
    } else {
      t = 0;
    }
    T = (bits >> 63) ? -(long long)t : (long long)t;
  }
#pragma unroll
  for (int i = 6; i > 0; --i) {
    const int d = (int)(((T + 128) & 255) - 128);
    out[i] = __float2bfloat16_rn((float)d);
    T = (T - d) >> 8;
  }
  out[0] = __float2bfloat16_rn((float)T);
}

// Tile images of the lower tiles (R, J), rbp <= J <= R < nrbt, of A (column-major, ld = n;
// diagonal tiles full), tile index f = (R - rbp)(R - rbp + 1)/2 + (J - rbp): one CTA per tile.
__global__ void __launch_bounds__(256) k_sv_digits(const double* __restrict__ A, int n, int rbp, uint8_t* img,
                                                   double* scl) {
  __shared__ double red[8];
  const long long f = blockIdx.x;
  int R, J;
  tile_of(f, rbp, R, J);
  const int t = threadIdx.x, r = t & 63, c0 = t >> 6;
  const int gr = R * TB + r;
  double v[16];
  double mx = 0.0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int gc = J * TB + c0 + 4 * k;
    v[k] = (gr < n && gc < n) ? A[gr + (long long)gc * n] : 0.0;
    mx = fmax(mx, fabs(v[k]));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((t & 31) == 0) red[t >> 5] = mx;
  __syncthreads();
  if (t < 32) {
    double m = (t < 8) ? red[t] : 0.0;
    for (int o = 4; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (t == 0) red[0] = m;
  }
  __syncthreads();
  const double u = fx_unit(red[0]);
  const double scale = 0x1p48 / u;
  uint8_t* base = img + f * (long long)SV_TILE;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    __nv_bfloat16 d[7];
    fx_digits<7>(v[k], scale, d);
    const int off = sv_sw(c0 + 4 * k, r);
#pragma unroll
    for (int q = 0; q < 7; ++q) *(__nv_bfloat16*)(base + q * SV_PLANE + off) = d[q];
  }
  if (t == 0) scl[f] = u;
}

template <int MODE>
__global__ void __launch_bounds__(RT, MODE == kPanelTc ? 1 : 2) k_panel(PanelParams p) {
  // mat-vec of P2: float64 register tiles, tensor cores from 7-digit images, or integer
  // multiply-adds from 53-bit images
  constexpr bool TC = MODE == kPanelTc;
  constexpr bool IX = MODE == kPanelInt;
  // the thread that arrives at the grid barriers: with the tensor-core mat-vec one of an
  // idle warp (warp 3), not the bulk-copy producer, whose fences would also wait for its
  // copies' bookkeeping
  constexpr int kLeader = TC ? 96 : 0;
  __shared__ double sh[kShBuf + RT];
  __shared__ double Wi[NBP], Vi[NBP], vtv[NBP], wtv[NBP];
  __shared__ __align__(16) double tile_s[TC ? 1 : TB * (TB + 1)];   // P1 scratch; P2 row-block sums [8][64]
  // tensor-core mat-vec: a ring of stages (tile image, x_J and x_R digits) in dynamic
  // shared memory, whose first stage doubles as P1's scratch (the phases never overlap)
  extern __shared__ uint8_t sv_raw[];
  __shared__ uint64_t sv_full[SV_STAGES], sv_empty[SV_STAGES], sv_accf[2], sv_acce[2], sv_drain;
  __shared__ float sv_xchg[TC ? 2 * 2 * 32 * 16 : 1];   // odd-digit partial levels, [tile parity][pair][lane][16]
  __shared__ uint32_t sv_tbase;
  __shared__ int sv_abort;
  uint8_t* sv_stages = TC ? (uint8_t*)(((uintptr_t)sv_raw + 1023) & ~(uintptr_t)1023) : nullptr;
  double* tile = TC ? (double*)sv_stages : tile_s;
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
  if constexpr (TC) {
    if (t == 0) {
      for (int s = 0; s < SV_STAGES; ++s) {
        sv_mbar_init(&sv_full[s], 2);    // the producer's expect-tx arrival and its x-digits arrival
        sv_mbar_init(&sv_empty[s], 1);
      }
      for (int b = 0; b < 2; ++b) {
        sv_mbar_init(&sv_accf[b], 1);
        sv_mbar_init(&sv_acce[b], 4);    // one arrival per epilogue warp
      }
      sv_mbar_init(&sv_drain, 1);
      sv_abort = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((t >> 5) == 2) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sv_u32(&sv_tbase)),
                   "r"(SV_TMEM) : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  long long sv_it = 0;       // tiles this CTA has taken through the tensor-core mat-vec
  bool aborted = false;
  // integer mat-vec: the common grid of the row sums, 2^(ix_ref - 52) (times 2^(e_x))
  int ix_ref = 0;
  double ix_unit = 0.0;
  if constexpr (IX) {
    ix_ref = grid_exp(__longlong_as_double((long long)*p.ix_gmax)) - 56;
    ix_unit = pow2i(ix_ref - 52);
  }

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
      const bool act = r < n;
      double upd = 0.0, wcorr = 0.0;
      double vs[NBP / 8], ws[NBP / 8];
      if (act && j > 0)
        wcorr = ldg_cg(p.Wp + r + (long long)(j - 1) * ld) + alpha_w * ldg_cg(A + r + (long long)(i - 1) * ld);
      // k < ceil(j / 8) (the same in every lane): groups with no column below j cost
      // no float64 instructions (the pipe spends one issue per warp instruction, however
      // many lanes take part)
      const int kj = (j + 7) >> 3;
#pragma unroll
      for (int k = 0; k < NBP / 8; ++k) {
        vs[k] = 0.0;
        ws[k] = 0.0;
      }
#pragma unroll
      for (int k = 0; k < NBP / 8; ++k) {
        if (k >= kj) break;
        const int c = q8 + 8 * k;
        if (act && c < j) {
          vs[k] = ldg_cg(A + r + (long long)(k0 + c) * ld);
          ws[k] = (c == j - 1) ? wcorr : ldg_cg(p.Wp + r + (long long)c * ld);
          upd += vs[k] * Wi[c] + ws[k] * Vi[c];
        }
      }
      upd += __shfl_xor_sync(0xffffffffu, upd, 1);
      upd += __shfl_xor_sync(0xffffffffu, upd, 2);
      upd += __shfl_xor_sync(0xffffffffu, upd, 4);
      double a = 0.0;
      if (act) a = ldg_cg(A + r + (long long)i * ld) - upd;
      double sq = 0.0;
      if (act && q8 == 0) {
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
      const double aa = (act && r >= i + 2) ? a : 0.0;
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
      if constexpr (TC || IX) {
        // largest |x_r| over the chunk's rows r >= i+1 (the scale of x's digits in P2)
        double mx = (act && r >= i + 1 && q8 == 0) ? fabs(a) : 0.0;
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
        if ((t & 31) == 0) sh[t >> 5] = mx;
        __syncthreads();
        if (t == 0) {
          double m = 0.0;
          for (int w2 = 0; w2 < RT / 32; ++w2) m = fmax(m, sh[w2]);
          p.sv_mx[ch] = m;
        }
        __syncthreads();
      }
    }
    if (!grid_sync(p.bar, p.status, epoch, p.spin_limit, kLeader)) { aborted = true; break; }
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
      if constexpr (IX) {
        // the same elements from the integer image (bit patterns held in float64 registers)
        const int rbi = k0 / TB;
        const long long fp = (long long)(R - rbi) * (R - rbi + 1) / 2 + (J - rbi);
        const double* tb = reinterpret_cast<const double*>(p.ix_img + fp * (TB * TB));
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) nxt[4 * c + k] = __ldca(tb + (cq0 + c) * TB + rq + 16 * k);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int gc = J * TB + cq0 + c;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int gr = R * TB + rq + 16 * k;
            nxt[4 * c + k] = (gr < n && gc < n) ? __ldca(A + gr + (long long)gc * ld) : 0.0;
          }
        }
      }
    };
    // the reflector's partials are loaded before the first tile, which would queue ahead of them
    const double ss0 = (t < n1) ? ldg_cg(p.p_ss + t) : 0.0;
    const long long mx0 = ((TC || IX) && t < n1) ? __double_as_longlong(ldg_cg(p.sv_mx + t)) : 0;
    asm volatile("" ::: "memory");
    if (f0 < f1) {
      tile_of(f0, rb0, R0, J0);
      if constexpr (!TC) load_tile(R0, J0);
    }
    double xmax = 0.0;
    const Refl h = householder(p, n1, sh, ss0, mx0, (TC || IX) ? &xmax : nullptr);
    const int ixe = IX ? grid_exp(xmax) : 0;   // integer mat-vec: |x| < 2^ixe
    {
      // V^T v = V(i+1,:) + scale * (sum over the P1 chunks), the same for W^T v:
      // these 2j sums are finished for P3 by one warp each, spread over the CTAs (warp 0
      // of CTA c first) so that no SM's float64 pipe takes more than one or two of them
      const int c = blockIdx.x + gridDim.x * wq;
      if (c < 2 * j) {
        // eight loads in flight per lane, added in ascending chunk order
        double s2 = 0.0;
        for (int ch0 = lane; ch0 < n1; ch0 += 32 * 8) {
          double v8[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int ch = ch0 + 32 * u;
            v8[u] = (ch < n1) ? ldg_cg(p.p_vw + (long long)ch * (2 * NBP) + c) : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) s2 += v8[u];
        }
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) {
          const double row1 = (c < j) ? ldg_cg(A + lo + (long long)(k0 + c) * ld) : ldg_cg(p.Wp + lo + (long long)(c - j) * ld);
          p.vwf[c] = row1 + h.scale * s2;
        }
      }
    }
    if constexpr (TC) {
      // Roles: warp 0 feeds the stages (bulk copies of tile images, x digits written by
      // the warp), one thread of warp 1 issues the MMAs, warps 4-7 drain the accumulators
      // (TMEM lane quadrant = warp % 4; with M = 64, row m sits in lane 32 (m/16) + m%16).
      volatile int* abort = &sv_abort;
      const int rbp = k0 / TB;
      const double ux = fx_unit(xmax);
      int xe = 0;                     // ux = 2^(xe - 7)
      frexp(ux, &xe);
      xe += 6;
      const long long nt = f1 - f0;
      // P1's generic-proxy use of the first stage is complete before the copy engine
      // writes the stages again
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (nt > 0 && wq == 0) {
        int R = R0, J = J0;
        long long issued = 0;
        // Lanes take elements lane and lane + 32 of a 64-block.  x_J's values are loaded one
        // tile ahead; x_R's digits are kept for the whole row block and written to every
        // stage that needs them.
        auto xval = [&](int B, int e2) {
          const int r = B * TB + lane + 32 * e2;
          return (r >= lo && r < n) ? ldg_cg(A + r + (long long)i * ld) : 0.0;
        };
        __nv_bfloat16 dr[2][7];
        int r_cached = -1;
        double xnJ[2] = {xval(J, 0), xval(J, 1)};
        double xnR[2] = {xval(R, 0), xval(R, 1)};
        for (long long q = 0; q < nt; ++q) {
          const long long it = sv_it + q;
          const int s = (int)(it % SV_STAGES);
          int ok = 1;
          if (lane == 0 && it >= SV_STAGES) ok = sv_wait(&sv_empty[s], (uint32_t)(((it / SV_STAGES) + 1) & 1), abort);
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (!ok) {
            if (lane == 0) { set_status(p.status, MOLGW_E_TIMEOUT); *abort = 1; atomicExch(&p.bar->abort, 1); }
            break;
          }
          uint8_t* st = sv_stages + (size_t)s * SV_STAGE;
          if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sv_u32(&sv_full[s])),
                         "r"(SV_TILE) : "memory");
          if (lane < 7) {
            // one copy per digit plane (8 KB each, concurrent), all completing on full[s]
            const long long fp = (long long)(R - rbp) * (R - rbp + 1) / 2 + (J - rbp);
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             sv_u32(st + lane * SV_PLANE)),
                         "l"(p.sv_img + fp * SV_TILE + lane * SV_PLANE), "r"(SV_PLANE), "r"(sv_u32(&sv_full[s]))
                         : "memory");
          }
          ++issued;
          const double xj[2] = {xnJ[0], xnJ[1]};
          if (R != r_cached) {
            // a new row block: the digits of x_R (its values were loaded ahead)
#pragma unroll
            for (int e2 = 0; e2 < 2; ++e2) sv_digits7(xnR[e2], xe, dr[e2]);
            r_cached = R;
          }
          int Rn = R, Jn = J + 1;
          if (Jn > Rn) { ++Rn; Jn = rb0; }
          if (q + 1 < nt) {
            xnJ[0] = xval(Jn, 0);
            xnJ[1] = xval(Jn, 1);
            if (Rn != R) {
              xnR[0] = xval(Rn, 0);
              xnR[1] = xval(Rn, 1);
            }
          }
          uint8_t* xi = st + SV_TILE;
#pragma unroll
          for (int e2 = 0; e2 < 2; ++e2) {
            const int e = lane + 32 * e2;
            __nv_bfloat16 d[7];
            sv_digits7(xj[e2], xe, d);
#pragma unroll
            for (int qd = 0; qd < 7; ++qd) *(__nv_bfloat16*)(xi + sv_sw(qd, e)) = d[qd];
            *(__nv_bfloat16*)(xi + sv_sw(7, e)) = __float2bfloat16_rn(0.0f);
            if (J < R) {
#pragma unroll
              for (int qd = 0; qd < 7; ++qd) *(__nv_bfloat16*)(xi + SV_XIMG + sv_sw(qd, e)) = dr[e2][qd];
              *(__nv_bfloat16*)(xi + SV_XIMG + sv_sw(7, e)) = __float2bfloat16_rn(0.0f);
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sv_u32(&sv_full[s])) : "memory");
          R = Rn;
          J = Jn;
        }
        // on an error path copies may still be in flight: they land before the phase ends
        if (lane == 0) {
          for (long long q = (issued > SV_STAGES ? issued - SV_STAGES : 0); q < issued; ++q) {
            const long long it = sv_it + q;
            for (long long k = 0; k < SV_SPIN; ++k)
              if (sv_mbar_try(&sv_full[it % SV_STAGES], (uint32_t)((it / SV_STAGES) & 1))) break;
          }
        }
        __syncwarp();
      } else if (nt > 0 && wq == 1) {
        if (lane == 0) {
          // D F32 (bit 4), A and B BF16 (bits 7, 10), A MN-major (bit 15) for A_RJ x_J,
          // N = 8 (N >> 3 at bit 17), M = 128 (M >> 4 at bit 24)
          const uint32_t id_n = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 17) | (8u << 24);
          const uint32_t id_t = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 17) | (8u << 24);
          int R = R0, J = J0;
          long long q = 0;
          for (; q < nt; ++q) {
            const long long it = sv_it + q;
            const int s = (int)(it % SV_STAGES), b = (int)(it & 1);
            if (!sv_wait(&sv_full[s], (uint32_t)((it / SV_STAGES) & 1), abort)) break;
            if (it >= 2 && !sv_wait(&sv_acce[b], (uint32_t)(((it >> 1) + 1) & 1), abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint8_t* st = sv_stages + (size_t)s * SV_STAGE;
            const uint32_t d0 = sv_tbase + (uint32_t)(b * 64);
            // Digit pair g = planes (2g, 2g+1) (the 4th pair's second plane lies past the
            // image and is discarded).  MN-major: the pair's 64-element atoms 8 KB apart
            // (leading byte offset), 8-row K groups 1 KB apart; K-major: 128 rows of 128 B.
            // Offsets move the start address (16-byte units: a pair 1024, a 16-row K step of
            // the MN-major operand 128, a 32-byte K step of a K-major one 2).
            const uint64_t a_mn = sv_desc(st, SV_PLANE, 1024), a_k = sv_desc(st, 16, 1024);
            const uint64_t bxj = sv_desc(st + SV_TILE, 16, 1024), bxr = sv_desc(st + SV_TILE + SV_XIMG, 16, 1024);
            const bool below = J < R;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
              for (int g = 0; g < 4; ++g) {
                sv_mma(d0 + 8 * g, a_mn + (uint64_t)(1024 * g + 128 * ks), bxj + (uint64_t)(2 * ks), id_n,
                       ks > 0 ? 1u : 0u);
                if (below)
                  sv_mma(d0 + 32 + 8 * g, a_k + (uint64_t)(1024 * g + 2 * ks), bxr + (uint64_t)(2 * ks), id_t,
                         ks > 0 ? 1u : 0u);
              }
            }
            sv_commit(&sv_empty[s]);
            sv_commit(&sv_accf[b]);
            if (++J > R) { ++R; J = rb0; }
          }
          if (q < nt) {
            set_status(p.status, MOLGW_E_TIMEOUT);
            *abort = 1;
            atomicExch(&p.bar->abort, 1);
            if (q > 0) {
              // the MMAs already issued finish before TMEM or the stages are given up
              sv_commit(&sv_drain);
              for (long long k = 0; k < SV_SPIN; ++k)
                if (sv_mbar_try(&sv_drain, 0u)) break;
            }
          }
        }
        __syncwarp();
      } else if (nt > 0 && wq >= 4) {
        // TMEM lane quadrant qd: warps qd = 0, 1 hold the even digits of tile rows 32 qd + lane,
        // warps qd = 2, 3 the odd digits of rows 32 (qd - 2) + lane
        const int qd = wq - 4;
        const bool odd = qd >= 2;
        const int pair = qd & 1;
        const int row = 32 * pair + lane;
        int R = R0, J = J0;
        double acc = 0.0;
        // tile scales, loaded one tile ahead
        double us_next = p.sv_scl[(long long)(R - rbp) * (R - rbp + 1) / 2 + (J - rbp)];
        // partial level sums of this warp's digits: l = i + j <= 6, i = 2g (+1 if odd)
        auto levels = [&](const uint32_t* S, float* P) {
#pragma unroll
          for (int l = 0; l < 7; ++l) P[l] = 0.0f;
#pragma unroll
          for (int g = 0; g < 4; ++g)
#pragma unroll
            for (int j = 0; j < 7; ++j) {
              const int l = 2 * g + j + (odd ? 1 : 0);
              if (l <= 6) P[l] += __uint_as_float(S[8 * g + j]);
            }
        };
        // value = (2^-24 vh + 2^-48 vl) u_tile u_x: two conversions, one multiply, one FMA
        auto finish = [&](const float* P, const float* Q, double us24) {
          long long L[7];
#pragma unroll
          for (int l = 0; l < 7; ++l) L[l] = __float2int_rn(P[l] + Q[l]);   // integers below 2^23: exact
          const long long vh = (L[0] << 24) + (L[1] << 16) + (L[2] << 8) + L[3];
          const long long vl = (L[4] << 16) + (L[5] << 8) + L[6];
          return fma((double)vl, us24 * 0x1p-24, (double)vh * us24);
        };
        for (long long q = 0; q < nt; ++q) {
          const long long it = sv_it + q;
          const int b = (int)(it & 1);
          int got = 1;
          if (lane == 0) got = sv_wait(&sv_accf[b], (uint32_t)((it >> 1) & 1), abort);
          got = __shfl_sync(0xffffffffu, got, 0);
          // the four epilogue warps agree (barrier 1 with an AND): a wait that ran out in one
          // of them ends the loop in all, so that their named barriers stay matched
          int all;
          asm volatile("{\n .reg .pred pi, po;\n setp.ne.s32 pi, %1, 0;\n bar.red.and.pred po, 1, 128, pi;\n selp.s32 %0, 1, 0, po;\n}"
                       : "=r"(all) : "r"(got) : "memory");
          if (!all) {
            if (lane == 0) { set_status(p.status, MOLGW_E_TIMEOUT); *abort = 1; atomicExch(&p.bar->abort, 1); }
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const bool below = J < R;
          const uint32_t tq = sv_tbase + ((uint32_t)(32 * qd) << 16) + (uint32_t)(b * 64);
          float Pn[7], Pt[7];
          {
            uint32_t S[32];
            sv_ld32(tq, S);                      // A_RJ x_J: columns 0..31 of the buffer
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            levels(S, Pn);
            if (below) {
              sv_ld32(tq + 32, S);               // A_RJ^T x_R: columns 32..63
              asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
              levels(S, Pt);
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sv_u32(&sv_acce[b])) : "memory");
          const double us = us_next * ux;
          {
            int Rn = R, Jn = J + 1;
            if (Jn > Rn) { ++Rn; Jn = rb0; }
            if (q + 1 < nt) us_next = p.sv_scl[(long long)(Rn - rbp) * (Rn - rbp + 1) / 2 + (Jn - rbp)];
          }
          float* xb = sv_xchg + ((q & 1) * 2 + pair) * 32 * 16 + lane * 16;
          // the even-digit warps hand their partial levels over; the odd-digit warps (on the
          // SM sub-partitions that neither the producer nor the MMA thread uses) finish
          if (!odd) {
#pragma unroll
            for (int l = 0; l < 7; ++l) {
              xb[l] = Pn[l];
              xb[8 + l] = below ? Pt[l] : 0.0f;
            }
          }
          asm volatile("bar.sync 1, 128;" ::: "memory");   // the four epilogue warps
          if (odd) {
            float Qn[7], Qt[7];
#pragma unroll
            for (int l = 0; l < 7; ++l) {
              Qn[l] = xb[l];
              Qt[l] = xb[8 + l];
            }
            acc += finish(Pn, Qn, us * 0x1p-24);
            if (below) {
              const long long ft = (long long)(R - rb0) * (R - rb0 + 1) / 2 + (J - rb0);
              p.p_t[ft * TB + row] = finish(Pt, Qt, us * 0x1p-24);
            }
            if (q + 1 == nt || J == R) {
              const int gr = R * TB + row;
              if (gr < n) p.p_y[(long long)blockIdx.x * n + gr] = acc;
              acc = 0.0;
            }
          }
          if (++J > R) { ++R; J = rb0; }
        }
      }
      sv_it += nt;
    } else if constexpr (IX) {
      if (f0 < f1) {
        const int rbi = k0 / TB;
        // x on its grid, m_x = rint(x 2^(53 - e_x)) = h 2^27 + l, each value converted by
        // one lane and handed to the lanes that use it by shuffles (x written by P1: read
        // through L2; the next tile's values are loaded with the tile)
        auto xv = [&](int r) { return (r >= lo && r < n) ? ldg_cg(A + r + (long long)i * ld) : 0.0; };
        auto xdig = [&](double v, int& h, int& l) { split27(fixed_round(v, 53 - ixe), h, l); };
        // y_R partials of the thread's rows on the common grid, 128-bit
        __int128 acc[4] = {0, 0, 0, 0};
        // x_R: lane converts rows lane and lane + 32 of the block, thread row rq + 16 k
        // comes from lane (rq + 16 k) mod 32
        int xrh[4], xrl[4];
        auto load_xr = [&](int R) {
          int h0, l0, h1, l1;
          xdig(xv(R * TB + lane), h0, l0);
          xdig(xv(R * TB + lane + 32), h1, l1);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int src = (rq + 16 * k) & 31;
            xrh[k] = __shfl_sync(0xffffffffu, k < 2 ? h0 : h1, src);
            xrl[k] = __shfl_sync(0xffffffffu, k < 2 ? l0 : l1, src);
          }
        };
        int R = R0, J = J0;
        load_xr(R);
        // x_J: lane converts column 8 wq + (lane & 7); thread column cq0 + c comes from
        // lane 4 (lane >> 4) + c
        double xj_next = xv(J * TB + 8 * wq + (lane & 7));
        for (long long f = f0; f < f1; ++f) {
          int Rn = R, Jn = J + 1;             // next tile
          if (Jn > Rn) { ++Rn; Jn = rb0; }
          int ah[16], al[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const long long w = __double_as_longlong(nxt[e]);
            al[e] = (int)(unsigned int)(unsigned long long)w;
            ah[e] = (int)(w >> 32);
          }
          int xch[4], xcl[4];
          {
            int h, l;
            xdig(xj_next, h, l);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              xch[c] = __shfl_sync(0xffffffffu, h, 4 * (lane >> 4) + c);
              xcl[c] = __shfl_sync(0xffffffffu, l, 4 * (lane >> 4) + c);
            }
          }
          if (f + 1 < f1) {
            load_tile(Rn, Jn);                // in flight while this tile is used
            xj_next = xv(Jn * TB + 8 * wq + (lane & 7));
          }
          const int sft = __ldg(p.ix_texp + ((long long)(R - rbi) * (R - rbi + 1) / 2 + (J - rbi))) - ix_ref;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            long long H = 0, M = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              H = mad_wide(ah[4 * c + k], xch[c], H);
              M = mad_wide(ah[4 * c + k], xcl[c], M);
              M = mad_wide(al[4 * c + k], xch[c], M);
            }
            const long long T = H + ((M + (1LL << 26)) >> 27);   // middle term rounded, not floored
            add_shifted(acc[k], T, sft);
          }
          if (J < R) {
            long long q[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              long long H = 0, M = 0;
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                H = mad_wide(ah[4 * c + k], xrh[k], H);
                M = mad_wide(ah[4 * c + k], xrl[k], M);
                M = mad_wide(al[4 * c + k], xrh[k], M);
              }
              q[c] = H + ((M + (1LL << 26)) >> 27);
            }
            // sums over the half-warp (the tile's 64 rows) scattering the four columns as
            // in the float64 path, in 64-bit integers (at most 2^59 in magnitude)
            const bool b3 = (rq & 8) != 0, b2 = (rq & 4) != 0;
            const long long k0v = b3 ? q[2] : q[0], k1v = b3 ? q[3] : q[1];
            const long long s0v = b3 ? q[0] : q[2], s1v = b3 ? q[1] : q[3];
            const long long h0 = k0v + __shfl_xor_sync(0xffffffffu, s0v, 8);
            const long long h1 = k1v + __shfl_xor_sync(0xffffffffu, s1v, 8);
            long long v = (b2 ? h1 : h0) + __shfl_xor_sync(0xffffffffu, b2 ? h0 : h1, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            if ((rq & 3) == 0) {
              const long long ft = (long long)(R - rb0) * (R - rb0 + 1) / 2 + (J - rb0);
              reinterpret_cast<long long*>(p.p_t)[ft * TB + cq0 + 2 * (b3 ? 1 : 0) + (b2 ? 1 : 0)] = v;
            }
          }
          if (f + 1 == f1 || J == R) {
            // end of this CTA's part of row block R: 128-bit sums over the 16 threads that
            // hold each row (the two half-warps, then the eight warps through shared memory),
            // rounded once to float64 from the common grid
            __int128* red = reinterpret_cast<__int128*>(tile);   // [8][64]
            __int128 a2[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              a2[k] = acc[k];
              const long long lo64 = (long long)(unsigned long long)a2[k];
              const long long hi64 = (long long)(a2[k] >> 64);
              const unsigned long long olo = (unsigned long long)__shfl_xor_sync(0xffffffffu, lo64, 16);
              const long long ohi = __shfl_xor_sync(0xffffffffu, hi64, 16);
              a2[k] += ((__int128)ohi << 64) | (__int128)olo;
            }
            __syncthreads();
            if (lane < 16) {
#pragma unroll
              for (int k = 0; k < 4; ++k) red[wq * TB + rq + 16 * k] = a2[k];
            }
            __syncthreads();
            if (t < TB) {
              __int128 y = red[t];
#pragma unroll
              for (int w2 = 1; w2 < RT / 32; ++w2) y += red[w2 * TB + t];
              const int r = R * TB + t;
              if (r < n) p.p_y[(long long)blockIdx.x * n + r] = i128_to_f64(y) * ix_unit * pow2i(ixe);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] = 0;
            if (f + 1 < f1 && Rn != R) load_xr(Rn);
          }
          R = Rn;
          J = Jn;
        }
      }
    } else {
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
    }
    if (!grid_sync(p.bar, p.status, epoch, p.spin_limit, kLeader)) { aborted = true; break; }

    // ---------------- P3: W column ----------------
    const int n3 = ceil_div_d(n - i - 1, RC);
    for (int c = t; c < 2 * j; c += blockDim.x) {
      const double v = ldg_cg(p.vwf + c);
      if (c < j) vtv[c] = v; else wtv[c - j] = v;
    }
    __syncthreads();
    for (int ch = L; ch < n3; ch += gridDim.x) {
      const int r = lo + ch * RC + rl;
      const bool act = r < n;
      double y = 0.0;
      if (act) {
        // (A22 x)_r = (direct partials of the CTAs whose ranges cover row block R)
        //           + (transposed partials of the tiles (R', R) below it);
        // y_r = scale (A22 x)_r + (1 - scale alpha) A(r, i+1) - W(r,:) V^T v - V(r,:) W^T v
        const int Rr = r / TB, a = Rr - rb0;
        const long long T = (long long)nrb * (nrb + 1) / 2;
        const long long fa = (long long)a * (a + 1) / 2, fb = fa + a;
        const int ca = (int)(((fa + 1) * gridDim.x - 1) / T), cb = (int)(((fb + 1) * gridDim.x - 1) / T);
        double yx = 0.0;
        // integer mat-vec: the transposed partials (units 2^(e_T - 52 + e_x), below 2^59)
        // moved to the common grid by left shifts (exact) and added in 128 bits
        __int128 yxi = 0;
        for (int c = ca + q8; c <= cb; c += 8) {
          // CTAs with an empty tile range wrote nothing
          if ((long long)c * T / gridDim.x == (long long)(c + 1) * T / gridDim.x) continue;
          yx += ldg_cg(p.p_y + (long long)c * n + r);
        }
#pragma unroll 8
        for (int R2 = Rr + 1 + q8; R2 < nrbt; R2 += 8) {
          const long long ft = (long long)(R2 - rb0) * (R2 - rb0 + 1) / 2 + a;
          if constexpr (IX) {
            const long long v = __ldcg(reinterpret_cast<const long long*>(p.p_t) + ft * TB + (r - Rr * TB));
            const int rbi = k0 / TB;
            const int sft = __ldg(p.ix_texp + ((long long)(R2 - rbi) * (R2 - rbi + 1) / 2 + (Rr - rbi))) - ix_ref;
            add_shifted(yxi, v, sft);
          } else {
            yx += ldg_cg(p.p_t + ft * TB + (r - Rr * TB));
          }
        }
        if constexpr (IX) yx = fma(i128_to_f64(yxi) * ix_unit, pow2i(ixe), yx);   // powers of two: exact scalings
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
      if (act && q8 == 0) {
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
    if (!grid_sync(p.bar, p.status, epoch, p.spin_limit, kLeader)) { aborted = true; break; }
  }

  // ---------------- end of panel: last W correction and packing ----------------
  if (!aborted) {
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
  if constexpr (TC) {
    // every role has finished (its MMAs and copies waited for) before TMEM is released
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((t >> 5) == 2) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sv_tbase), "r"(SV_TMEM) : "memory");
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
int g_sv_blocks_per_sm = -1;     // k_panel<kPanelTc>: co-resident CTAs per SM with its stage ring (0: unusable)
int g_ix_blocks_per_sm = -1;     // k_panel<kPanelInt>: co-resident CTAs per SM
constexpr int kSvMinRows = 1024; // trailing matrices from this size use the tensor-core mat-vec
constexpr int kIxMinRows = 256;  // and the integer one

}  // namespace

int tridiag_coop_capacity() {
  if (g_coop_blocks_per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_panel<kPanelF64>, RT, 0);
    g_coop_blocks_per_sm = std::max(1, std::min(occ, 2));
    g_coop_blocks_per_sm = std::min(g_coop_blocks_per_sm, kMaxPanelGrid / std::max(g_num_sms, 1));
    int occ_sv = 0;
    if (cudaFuncSetAttribute(k_panel<kPanelTc>, cudaFuncAttributeMaxDynamicSharedMemorySize, SV_SMEM) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_sv, k_panel<kPanelTc>, RT, SV_SMEM) == cudaSuccess)
      g_sv_blocks_per_sm = std::min(occ_sv, 1);
    else
      g_sv_blocks_per_sm = 0;
    int occ_ix = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_ix, k_panel<kPanelInt>, RT, 0) == cudaSuccess)
      g_ix_blocks_per_sm = std::min(std::min(occ_ix, 2), kMaxPanelGrid / std::max(g_num_sms, 1));
    else
      g_ix_blocks_per_sm = 0;
    cudaGetLastError();
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
  // Tensor-core mat-vec (MOLGW_FLAG_EIG_TC, the context's own stream): tile images and
  // scales in w.sv, then the column-maximum partials.
  // Integer mat-vec (the same arena: 32 KB images, the tiles' exponents where the tile
  // scales are, the largest |a| after the column-maximum partials).  Which one
  // runs: ex.panel_matvec (MOLGW_MATVEC_*), automatic = the integer one.
  // The tensor-core one only on the context's own stream (one CTA per SM and TMEM); the
  // integer one on concurrent lanes too, with the lane's share of the co-resident CTAs.
  const bool arena = w.sv && n <= w.sv_n;
  const int want = ex.panel_matvec;
  const bool sv_ok = arena && ex.coop_cap == 0 && g_sv_blocks_per_sm > 0 && want == MOLGW_MATVEC_TC;
  const bool ix_ok = arena && g_ix_blocks_per_sm > 0 && (want == MOLGW_MATVEC_AUTO || want == MOLGW_MATVEC_INT);

  if (arena) {
    const long long cap_tiles = eig_sv_tiles(w.sv_n);
    p.sv_img = (const uint8_t*)w.sv;
    p.sv_scl = (const double*)((uint8_t*)w.sv + cap_tiles * kSvTileBytes);
    p.sv_mx = (double*)p.sv_scl + cap_tiles;
    p.ix_img = (const long long*)w.sv;
    p.ix_texp = (const int*)p.sv_scl;
    p.ix_gmax = (const unsigned long long*)(p.sv_mx + (w.sv_n + 31) / 32 + 2);
  }
  const int ncols = n - 1;
  for (int k0 = 0; k0 < ncols; k0 += NBP) {
    const int nbp = std::min(NBP, ncols - k0);
    const int k1 = k0 + nbp;
    p.k0 = k0; p.nbp = nbp; p.k1 = k1;
    const int nrb = nrbt - (k0 + 1) / TB;
    const long long tiles = (long long)nrb * (nrb + 1) / 2;
    if (ix_ok && n - k0 >= kIxMinRows) {
      KScope ks(ex, MOLGW_K_TRIDIAG_PANEL, 2);
      const int rbp = k0 / TB;
      const long long tiles_p = (long long)(nrbt - rbp) * (nrbt - rbp + 1) / 2;
      cudaMemsetAsync((void*)p.ix_gmax, 0, sizeof(unsigned long long), ex.st);
      k_ix_image<<<(unsigned)tiles_p, 256, 0, ex.st>>>(A, n, rbp, (long long*)p.ix_img, (int*)p.ix_texp,
                                                       (unsigned long long*)p.ix_gmax);
      int cap_ix = g_num_sms * g_ix_blocks_per_sm;
      if (ex.coop_cap > 0) cap_ix = std::max(2 * NBP / (RT / 32), std::min(cap_ix, ex.coop_cap));
      const int grid = (int)std::max<long long>(2 * NBP / (RT / 32),
                                                 std::min<long long>(cap_ix, std::max<long long>(tiles, ceil_div(n - k0, RC))));
      cudaMemsetAsync(p.bar, 0, sizeof(GridBar), ex.st);
      void* args[] = {&p};
      cudaLaunchCooperativeKernel((const void*)k_panel<kPanelInt>, dim3(grid), dim3(RT), args, 0, ex.st);
    } else if (sv_ok && n - k0 >= kSvMinRows) {
      KScope ks(ex, MOLGW_K_TRIDIAG_PANEL, 2);
      const int rbp = k0 / TB;
      const long long tiles_p = (long long)(nrbt - rbp) * (nrbt - rbp + 1) / 2;
      k_sv_digits<<<(unsigned)tiles_p, 256, 0, ex.st>>>(A, n, rbp, (uint8_t*)p.sv_img, (double*)p.sv_scl);
      const int cap_sv = g_num_sms * g_sv_blocks_per_sm;
      const int grid = (int)std::max<long long>(2 * NBP / (RT / 32),
                                                 std::min<long long>(cap_sv, std::max<long long>(tiles, ceil_div(n - k0, RC))));
      cudaMemsetAsync(p.bar, 0, sizeof(GridBar), ex.st);
      void* args[] = {&p};
      cudaLaunchCooperativeKernel((const void*)k_panel<kPanelTc>, dim3(grid), dim3(RT), args, SV_SMEM, ex.st);
    } else {
      const int grid = (int)std::max<long long>(2 * NBP / (RT / 32),
                                                 std::min<long long>(cap, std::max<long long>(tiles, ceil_div(n - k0, RC))));
      KScope ks(ex, MOLGW_K_TRIDIAG_PANEL, 1);
      cudaMemsetAsync(p.bar, 0, sizeof(GridBar), ex.st);
      void* args[] = {&p};
      cudaLaunchCooperativeKernel((const void*)k_panel<kPanelF64>, dim3(grid), dim3(RT), args, 0, ex.st);
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
