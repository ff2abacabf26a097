// Fixed-point split GEMM on the BF16 tensor cores with exact float32 sums.
//
// Every float64 value x of a row's group of kFxGroup consecutive K elements is
// written with NS base-256 digits: x ~ u * sum_i s_i 2^(-8i), where u = 2^(e-7)
// is one power of two for the (row, group) with max|x| < 2^e, and the digits s_i
// are the balanced base-256 digits of rint(2^(8(NS-1)) x / u), integers in
// [-128, 128] (exact in BF16).  A product of two digits is an integer below 2^14
// in magnitude; the products with i + j < NS are summed per "level" l = i + j in
// NS float32 accumulators over chunks of K elements short enough that every
// partial sum is an integer below 2^24, so the float32 accumulation is exact.
// The levels are combined exactly in 64-bit integers and only the result of a
// group is rounded, to float64.  The only approximation is the truncation of x
// to 8 NS bits relative to the largest |x| of its (row, group).
//   NS = 4 (MOLGW_PREC_BF16X10): 10 products, 32 bits, 256-element chunks;
//   NS = 7: 28 products, 56 bits -- every value within a factor 4 of its group's
//           largest is represented exactly, so the product matches float64
//           accuracy (normwise); 128-element chunks.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace molgw {

constexpr int kFxSlices = 4;       // digits of the BF16X10 precision
constexpr int kFxMaxSlices = 7;
constexpr int kFxKBlock = 64;      // K padding unit of every operand
constexpr int kFxGroup = 1024;     // K elements per scale u (one CTA's K range)

inline long long fx_pad(long long k) { return (k + kFxKBlock - 1) / kFxKBlock * kFxKBlock; }
inline int fx_groups(long long ld) { return (int)((ld + kFxGroup - 1) / kFxGroup); }

// rows x ld BF16 digits (ns of them; ld a multiple of kFxKBlock) and the float64
// scale u of each (row, group), at u[row * ngroups + group].
struct FxMat {
  void* s[kFxMaxSlices] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* u = nullptr;
  long long rows = 0, ld = 0;
  int ngroups = 0;
  int ns = kFxSlices;
};

// bytes of an FxMat of rows x ld (ld padded) with ns digits, 256-byte aligned parts
size_t fx_mat_bytes(long long rows, long long ld, int ns = kFxSlices);
// lay an FxMat out over device memory of fx_mat_bytes(rows, ld, ns) bytes
FxMat fx_mat_carve(void* base, long long rows, long long ld, int ns = kFxSlices);
// rows of an FxMat starting at row r0 (the same K layout)
FxMat fx_rows(const FxMat& m, long long r0, long long rows);

// C = A B^T over K (a multiple of kFxKBlock, <= A.ld, B.ld); A.ns == B.ns (4 or 7).
// The K range splits into groups of kFxGroup; group g of the CTA grid writes its
// float64 result to out + g * split_stride (one group: no partials).  Element
// (row, col) goes to out[row * out_ld + col], or out[col * out_ld + row] with
// col_major.  accumulate (one group only): out = out + alpha * C.  lower_only:
// only elements in 64 x 64 blocks on or below the diagonal (row/64 >= col/64).
struct FxGemm {
  int M = 0, N = 0, K = 0;
  int k0 = 0;                 // first K element (a multiple of kFxGroup)
  FxMat A, B;
  double* out = nullptr;
  long long out_ld = 0;
  long long split_stride = 0;
  bool col_major = false;
  bool accumulate = false;
  double alpha = 1.0;
  bool lower_only = false;
  const double* diag = nullptr;   // adds diag[row]^2 where row == col (not with accumulate)
  int kclass = MOLGW_K_GEMM_TC;   // kernel class for launch accounting
};
int fx_gemm(Exec& ex, const FxGemm& g);
// Arena of the 7-digit operands of the eigensolver (MOLGW_FLAG_EIG_TC) for
// matrices up to n and back-transformations of up to ncols columns: the two
// 128-wide SYR2K operands, or (later in the same solve) the back-transformation
// operands V^T, X^T, V, T-product and a block of kFxZBlock eigenvector columns.
constexpr int kFxZBlock = 2048;
inline size_t eig_fx_bytes(long long n, long long ncols) {
  const long long np = fx_pad(n);
  const size_t syr2k = 2 * fx_mat_bytes(n, 128, 7);
  const size_t bt = fx_mat_bytes(64, np, 7) + fx_mat_bytes(ncols, np, 7) + fx_mat_bytes(n, 64, 7) +
                    fx_mat_bytes(ncols, 64, 7) + fx_mat_bytes(n < kFxZBlock ? n : kFxZBlock, np, 7);
  return syr2k > bt ? syr2k : bt;
}

// number of K groups (= output splits) of a K range
inline int fx_nsplit(int K) { return (K + kFxGroup - 1) / kFxGroup; }

// ---------------------------------------------------------------------------
// The NS digits of y = x / u (|y| < 128): T = rint(y 2^(8(NS-1))) (one float64
// scaling, exact, and one rounding) split into balanced base-256 digits in
// [-128, 127] below a leading digit in [-128, 128], y ~ sum_i s_i 2^(-8i), with
// integer arithmetic (the float64 pipe does two operations per value).
// scale = 2^(8(NS-1)) / u.
template <int NS>
__device__ __forceinline__ void fx_digits(double x, double scale, __nv_bfloat16* out) {
  long long T = __double2ll_rn(x * scale);
#pragma unroll
  for (int i = NS - 1; i > 0; --i) {
    const int d = (int)(((T + 128) & 255) - 128);
    out[i] = __float2bfloat16_rn((float)d);
    T = (T - d) >> 8;
  }
  out[0] = __float2bfloat16_rn((float)T);
}

// u = 2^(e-7) for max |x| < 2^e (2^-7 for zero); scale24 = 2^24 / u
__device__ __forceinline__ double fx_unit(double maxabs) {
  int e = 0;
  if (maxabs > 0.0) frexp(maxabs, &e);
  return ldexp(1.0, e - 7);
}

// Slicing of any element source f(r, k) (a device functor returning a float64,
// zero outside the matrix): pass 1 finds the scale u of each (row, group), pass 2
// writes the four slices.  Reads go with lanes over rows (coalesced for sources
// stored row-fastest), writes with lanes along K.
// ---------------------------------------------------------------------------
constexpr int kFxTileK = 128;   // K elements per slicing tile (divides kFxGroup)

// u = 2^(e-7) with max |x| < 2^e over the row's group (2^-7 for an all-zero group)
template <class Src>
__global__ void k_fx_scale(Src f, long long rows, long long ld, FxMat dst) {
  __shared__ double red[8][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long r = (long long)blockIdx.x * 32 + lane;
  const long long k0 = (long long)blockIdx.y * kFxGroup;
  const long long k1 = (ld < k0 + kFxGroup) ? ld : k0 + kFxGroup;
  double m = 0.0;
  for (long long k = k0 + warp; k < k1; k += 8) m = fmax(m, fabs(f(r, k)));
  red[warp][lane] = m;
  __syncthreads();
  if (warp == 0 && r < rows) {
    for (int w = 1; w < 8; ++w) m = fmax(m, red[w][lane]);
    dst.u[r * dst.ngroups + blockIdx.y] = fx_unit(m);
  }
}

// the digits of a 32-row x kFxTileK tile
template <int NS, class Src>
__global__ void k_fx_slices(Src f, long long rows, long long ld, FxMat dst) {
  __shared__ double tile[kFxTileK][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long r0 = (long long)blockIdx.x * 32, c0 = (long long)blockIdx.y * kFxTileK;
  for (int k = warp; k < kFxTileK; k += 8) tile[k][lane] = (c0 + k < ld) ? f(r0 + lane, c0 + k) : 0.0;
  __syncthreads();
  const int g = (int)(c0 / kFxGroup);
  for (int rr = warp; rr < 32; rr += 8) {
    const long long r = r0 + rr;
    if (r >= rows) break;
    const double scale = ldexp(1.0, 8 * (NS - 1)) / dst.u[r * dst.ngroups + g];   // a power of two
#pragma unroll
    for (int j = 0; j < kFxTileK / 32; ++j) {
      const int k = lane + 32 * j;
      if (c0 + k < ld) {
        __nv_bfloat16 d[NS];
        fx_digits<NS>(tile[k][rr], scale, d);
        const long long o = r * dst.ld + c0 + k;
#pragma unroll
        for (int i = 0; i < NS; ++i) ((__nv_bfloat16*)dst.s[i])[o] = d[i];
      }
    }
  }
}

// For sources contiguous along K (src[r*sr + k], e.g. a row-major operand): one warp
// per (row, group), lanes along K, the group's maximum then its digits, both
// passes coalesced.
template <int NS>
__global__ void k_fx_rows(const double* __restrict__ src, long long rows, long long cols, long long sr,
                          const double* __restrict__ row_scale, FxMat dst) {
  const int lane = threadIdx.x & 31;
  const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long r = wg / dst.ngroups;
  const int g = (int)(wg % dst.ngroups);
  if (r >= rows) return;
  const long long k0 = (long long)g * kFxGroup;
  const long long k1 = (dst.ld < k0 + kFxGroup) ? dst.ld : k0 + kFxGroup;
  const double rs = row_scale ? row_scale[r] : 1.0;
  double m = 0.0;
  for (long long k = k0 + lane; k < k1; k += 32)
    if (k < cols) m = fmax(m, fabs(src[r * sr + k] * rs));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  const double u = fx_unit(m);
  if (lane == 0) dst.u[r * dst.ngroups + g] = u;
  const double scale = ldexp(1.0, 8 * (NS - 1)) / u;
  for (long long k = k0 + lane; k < k1; k += 32) {
    const double x = (k < cols) ? src[r * sr + k] * rs : 0.0;
    __nv_bfloat16 d[NS];
    fx_digits<NS>(x, scale, d);
#pragma unroll
    for (int i = 0; i < NS; ++i) ((__nv_bfloat16*)dst.s[i])[r * dst.ld + k] = d[i];
  }
}

template <class Src>
void fx_slice(Exec& ex, const Src& f, long long rows, FxMat dst, int kclass = MOLGW_K_MISC) {
  if (rows <= 0) return;
  KScope ks(ex, kclass, 2);
  dim3 g1(ceil_div(rows, 32), dst.ngroups);
  k_fx_scale<Src><<<g1, 256, 0, ex.st>>>(f, rows, dst.ld, dst);
  dim3 g2(ceil_div(rows, 32), ceil_div(dst.ld, kFxTileK));
  if (dst.ns == 7)
    k_fx_slices<7, Src><<<g2, 256, 0, ex.st>>>(f, rows, dst.ld, dst);
  else
    k_fx_slices<4, Src><<<g2, 256, 0, ex.st>>>(f, rows, dst.ld, dst);
}

struct FxStrided {
  const double* src;
  long long sr, sk, rows, cols;
  const double* row_scale;
  __device__ double operator()(long long r, long long k) const {
    if (r >= rows || k >= cols) return 0.0;
    const double v = src[r * sr + k * sk];
    return row_scale ? v * row_scale[r] : v;
  }
};

// Slice a strided float64 matrix: element (r, k) = src[r*sr + k*sk] for k < cols,
// zero for cols <= k < dst.ld; row_scale (optional) multiplies row r.
void fx_split(Exec& ex, const double* src, long long rows, long long cols, long long sr, long long sk,
              const double* row_scale, FxMat dst, int kclass = MOLGW_K_MISC);

// out[r][c] = beta*out[r][c] + sum_{s<ns} part[s][r][c]  (row-major partials)
void fx_reduce_rm(Exec& ex, const double* part, int ns, long long split_stride, int M, int N, double* out,
                  long long ldo, double beta);

// out[r][c] = beta*out[r][c] + sum_{s<ns} part[s][c][r]  (col-major partials)
void fx_reduce_cm(Exec& ex, const double* part, int ns, long long split_stride, int M, int N, double* out,
                  long long ldo, double beta);

}  // namespace molgw
