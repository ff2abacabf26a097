// Split-precision tensor-core GEMM engine (tcgen05 + TMEM + TMA) for sm_103a.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace molgw {

// Operand arithmetic of the tensor-core path.  Each float64 value x is split as
// x = hi + lo with hi = round(x) and lo = round(x - hi) in the operand format;
// a product is taken as hi*hi + hi*lo + lo*hi with FP32 accumulation (the lo*lo
// term is dropped).  BF16 keeps 8 significant bits per part (~16 in total), TF32
// keeps 11 (~22 in total).
// BF16X6 splits into three BF16 slices x = hi + mid + lo (~24 bits) and takes the
// six products hi*hi + hi*mid + mid*hi + hi*lo + mid*mid + lo*hi.
enum TcPrec { TC_BF16X3 = 0, TC_TF32X3 = 1, TC_BF16X6 = 2 };

inline int tc_elem_bytes(int prec) { return prec == TC_TF32X3 ? 4 : 2; }
inline int tc_slices(int prec) { return prec == TC_BF16X6 ? 3 : 2; }
// K (and padded row length) granularity in elements: one 128-byte swizzle row.
inline int tc_kblock(int prec) { return prec == TC_TF32X3 ? 32 : 64; }
inline long long tc_pad(long long k, int prec) { const int b = tc_kblock(prec); return (k + b - 1) / b * b; }

// A split operand: rows x ld elements (ld padded to tc_kblock), hi and lo parts
// (and lo2, the third slice of BF16X6).
struct TcMat {
  void* hi = nullptr;
  void* lo = nullptr;
  void* lo2 = nullptr;
  long long rows = 0, ld = 0;
};

enum TcEpi {
  TC_EPI_F32_PARTIAL = 0,  // out_f32[split][M][N]
  TC_EPI_SPLIT = 1,        // split result into out_split (row-major, ld = out_ld)
  TC_EPI_F64 = 2,          // out_f64[row * out_ld + col]
  TC_EPI_RPA = 3           // out_f64 column-major (n x n, lower tiles) + D_t^2 on the diagonal
};

struct TcEpilogue {
  int mode = TC_EPI_F32_PARTIAL;
  float* out_f32 = nullptr;
  double* out_f64 = nullptr;
  long long out_ld = 0;
  TcMat out_split;                 // TC_EPI_SPLIT
  const double* diag = nullptr;    // TC_EPI_RPA: D_t
};

struct TcGemm {
  int prec = TC_BF16X3;
  int M = 0, N = 0, K = 0;        // K: multiple of tc_kblock (operands zero-padded)
  TcMat A, B;                     // A: rows >= M (+ batch offsets), B: rows >= N
  int batch = 1;
  long long a_batch_rows = 0, b_batch_rows = 0, out_batch_rows = 0;  // per-batch row offsets
  int ksplit = 1;                 // TC_EPI_F32_PARTIAL only
  bool lower_only = false;        // only 128x128 output tiles with tile_row >= tile_col
  TcEpilogue epi;
};

int tc_gemm(Exec& ex, const TcGemm& g);

__device__ __forceinline__ uint32_t tc_f32_to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Store x as its (hi, lo) split at element idx of a split operand.
template <int PREC>
__device__ __forceinline__ void tc_store_split(const TcMat& m, long long idx, double x) {
  if (PREC == TC_BF16X3) {
    const __nv_bfloat16 h = __double2bfloat16(x);
    const __nv_bfloat16 l = __double2bfloat16(x - (double)__bfloat162float(h));
    ((__nv_bfloat16*)m.hi)[idx] = h;
    ((__nv_bfloat16*)m.lo)[idx] = l;
  } else if (PREC == TC_BF16X6) {
    const __nv_bfloat16 h = __double2bfloat16(x);
    const double r1 = x - (double)__bfloat162float(h);
    const __nv_bfloat16 md = __double2bfloat16(r1);
    const __nv_bfloat16 l = __double2bfloat16(r1 - (double)__bfloat162float(md));
    ((__nv_bfloat16*)m.hi)[idx] = h;
    ((__nv_bfloat16*)m.lo)[idx] = md;
    ((__nv_bfloat16*)m.lo2)[idx] = l;
  } else {
    const uint32_t h = tc_f32_to_tf32((float)x);
    const uint32_t l = tc_f32_to_tf32((float)(x - (double)__uint_as_float(h)));
    ((uint32_t*)m.hi)[idx] = h;
    ((uint32_t*)m.lo)[idx] = l;
  }
}
// Number of K splits tc_gemm uses for nkb K blocks and a requested split count.
int tc_ksplit_of(int nkb, int ks);

// Split a strided float64 matrix into a padded operand:
// dst[r][k] = split(scale_r * src[r*sr + k*sk]) for k < cols, zero for cols <= k < ld.
// row_scale (optional) multiplies row r.
void tc_split(Exec& ex, int prec, const double* src, long long rows, long long cols, long long sr, long long sk,
              const double* row_scale, TcMat dst);

// Sum of ksplit float32 partial M x N blocks into a float64 matrix with beta.
void tc_reduce_partials(Exec& ex, const float* part, int ksplit, int M, int N, double* out, long long ldo,
                        double beta);

}  // namespace molgw
