// Split-precision tensor-core GEMM on tcgen05 (sm_103a).
//
// D[M][N] = sum_k A[m][k] B[n][k] with A and B stored K-major (rows of K
// contiguous elements, zero-padded to a multiple of one 128-byte swizzle row).
// Every operand is a pair (hi, lo) of BF16 or TF32 values; the three products
// hi*hi + hi*lo + lo*hi accumulate in FP32 in tensor memory.
//
// One 128x128 output tile per CTA; 8 warps with fixed roles:
//   warp 0  TMA producer: 128B-swizzled 128 x (128 B) boxes of A_hi, A_lo, B_hi,
//           B_lo per K block into a 3-stage shared-memory ring (64 KB per stage);
//   warp 1  one thread issues the tcgen05.mma instructions (kind::f16 or
//           kind::tf32, M=128, N=128, 4 K-steps x 3 products per stage) and
//           commits each stage back to the producer through an mbarrier;
//   warp 2  allocates and frees the 128 TMEM columns of the accumulator;
//   warps 4-7 the epilogue: tcgen05.ld of its 32-lane quarter, then the mode's
//           store (float32 partials, split operands, float64, the RPA matrix with
//           its D^2 diagonal, or the self-energy w / g-weighted w).
// Every mbarrier wait is bounded; on a timeout the kernel latches
// MOLGW_E_TIMEOUT and still releases its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include "tc.cuh"

namespace molgw {

namespace {

constexpr int BM = 128, BN = 128, KROW = 128;          // tile rows, tile cols, bytes per K row
constexpr int TILE = BM * KROW;                        // 16 KB per operand tile
// per stage: the slices of A then the slices of B (4 tiles with 2 slices, 6 with 3)
template <int NS> struct Ring {
  static constexpr int STAGE = 2 * NS * TILE;
  static constexpr int STAGES = (NS == 2) ? 3 : 2;
  static constexpr int SMEM = STAGES * STAGE + 1024;
};
constexpr long long SPIN_LIMIT = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t cnt) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  const uint32_t a = smem_u32(b);
  for (long long it = 0; it < SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc_sw128(const void* p) {
  const uint32_t a = smem_u32(p);
  uint64_t d = (uint64_t)((a & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}
template <int PREC>
__device__ __forceinline__ void mma(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  if (PREC != TC_TF32X3)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}

struct KParams {
  int M, N, nkb, kchunk, batch, ksplit, lower_only;
  long long a_batch_rows, b_batch_rows, out_batch_rows;
  TcEpilogue epi;
  int* status;
};

template <int PREC>
__global__ void __launch_bounds__(256, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                   const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mB0,
                   const __grid_constant__ CUtensorMap mB1, const __grid_constant__ CUtensorMap mB2, KParams p) {
  constexpr int NS = (PREC == TC_BF16X6) ? 3 : 2;
  constexpr int STAGE = Ring<NS>::STAGE, STAGES = Ring<NS>::STAGES;
  const CUtensorMap* mapA[3] = {&mA0, &mA1, &mA2};
  const CUtensorMap* mapB[3] = {&mB0, &mB1, &mB2};
  const int bn = blockIdx.x, bm = blockIdx.y;
  if (p.lower_only && bm < bn) return;
  const int b = blockIdx.z % p.batch, kz = blockIdx.z / p.batch;
  const int kb0 = kz * p.kchunk, kb1 = min(p.nkb, kb0 + p.kchunk);
  const int nk = kb1 - kb0;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[3], empty[3], done, drain;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = bm * BM, n0 = bn * BN;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    mbar_init(&drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)), "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base;
  const int arow = (int)(b * p.a_batch_rows) + m0, brow = (int)(b * p.b_batch_rows) + n0;
  constexpr int KE = (PREC == TC_TF32X3) ? 32 : 64;     // elements per K block

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int i = 0; i < nk; ++i) {
      const int s = i % STAGES;
      if (i >= STAGES && !mbar_wait(&empty[s], ((i / STAGES) + 1) & 1)) {
        set_status(p.status, MOLGW_E_TIMEOUT);
        break;
      }
      uint8_t* st = smem + s * STAGE;
      mbar_expect_tx(&full[s], STAGE);
      const int x = (kb0 + i) * KE;
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        tma_load_2d(st + sl * TILE, mapA[sl], &full[s], x, arow);
        tma_load_2d(st + (NS + sl) * TILE, mapB[sl], &full[s], x, brow);
      }
      issued = i + 1;
    }
    // copies still in flight (only on an error path) land before the CTA leaves
    for (int i = (issued > STAGES ? issued - STAGES : 0); i < issued; ++i) mbar_wait(&full[i % STAGES], (i / STAGES) & 1);
  } else if (warp == 1 && lane == 0) {
    // D F32 (bit 4); A, B type at bits 7-9 / 10-12 (BF16 = 1, TF32 = 2); K-major; N>>3 at 17; M>>4 at 24
    const uint32_t ty = (PREC == TC_TF32X3) ? 2u : 1u;
    const uint32_t idesc = (1u << 4) | (ty << 7) | (ty << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    bool ok = true;
    int i = 0;
    for (; i < nk; ++i) {
      const int s = i % STAGES;
      if (!mbar_wait(&full[s], (i / STAGES) & 1)) {
        set_status(p.status, MOLGW_E_TIMEOUT);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint8_t* st = smem + s * STAGE;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {         // 4 x 32 bytes of K per 128-byte row
        const uint64_t o = 2 * kk;             // +32 B in the 16-byte-encoded address field
        // products of slices (a, b) with a + b < NS: hi*hi first
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
          for (int b = 0; a + b < NS; ++b) {
            const uint64_t ad = sdesc_sw128(st + a * TILE) + o, bd = sdesc_sw128(st + (NS + b) * TILE) + o;
            mma<PREC>(tbase, ad, bd, idesc, (i > 0 || kk > 0 || a > 0 || b > 0) ? 1u : 0u);
          }
      }
      mma_commit(&empty[s]);
    }
    if (ok) {
      mma_commit(&done);
    } else if (i > 0) {
      // error path: the MMAs already issued finish (bounded wait) before the CTA
      // releases TMEM
      mma_commit(&drain);
      mbar_wait(&drain, 0);
    }
  } else if (warp >= 4) {
    const int q = warp & 3;
    const bool ok = (nk > 0) ? mbar_wait(&done, 0) : true;
    if (!ok) set_status(p.status, MOLGW_E_TIMEOUT);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int lrow = 32 * q + lane;
    const int row = m0 + lrow;
    const TcEpilogue& e = p.epi;
    for (int c = 0; c < BN; c += 16) {
      uint32_t r[16];
      const uint32_t taddr = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)c;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (!ok || row >= p.M) continue;
#pragma unroll 4
      for (int jj = 0; jj < 16; ++jj) {
        const int col = n0 + c + jj;
        if (col >= p.N) break;
        const float v = (nk > 0) ? __uint_as_float(r[jj]) : 0.0f;
        switch (e.mode) {
          case TC_EPI_F32_PARTIAL:
            e.out_f32[((long long)kz * p.M + row) * p.N + col] = v;
            break;
          case TC_EPI_SPLIT:
            tc_store_split<PREC>(e.out_split, (b * p.out_batch_rows + row) * e.out_split.ld + col, (double)v);
            break;
          case TC_EPI_F64:
            e.out_f64[(b * p.out_batch_rows + row) * e.out_ld + col] = (double)v;
            break;
          case TC_EPI_RPA: {
            // column-major lower triangle (element (row, col) at col*ld + row): the
            // layout the tridiagonalisation reads; lanes of a warp hit consecutive rows
            double x = (double)v;
            if (row == col) x += e.diag[row] * e.diag[row];
            e.out_f64[(long long)col * e.out_ld + row] = x;
            break;
          }
          default:
            break;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(BN) : "memory");
  }
}

// ---------------------------------------------------------------------------
// splits, reductions
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void k_split(const double* __restrict__ src, long long rows, long long cols, long long sr, long long sk,
                        const double* __restrict__ row_scale, TcMat dst) {
  __shared__ double tile[32][33];
  const long long r0 = (long long)blockIdx.y * 32, k0 = (long long)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  const bool kfast = (sk == 1);
  for (int i = 0; i < 32; i += 8) {
    const long long r = r0 + (kfast ? ty + i : tx), k = k0 + (kfast ? tx : ty + i);
    double v = 0.0;
    if (r < rows && k < cols) {
      v = src[r * sr + k * sk];
      if (row_scale) v *= row_scale[r];
    }
    tile[(int)(r - r0)][(int)(k - k0)] = v;
  }
  __syncthreads();
  for (int i = 0; i < 32; i += 8) {
    const long long r = r0 + ty + i, k = k0 + tx;
    if (r < rows && k < dst.ld) tc_store_split<PREC>(dst, r * dst.ld + k, tile[ty + i][tx]);
  }
}

__global__ void k_reduce_partials(const float* __restrict__ part, int ksplit, int M, int N, double* out, long long ldo,
                                  double beta) {
  const long long total = (long long)M * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < ksplit; ++k) s += (double)part[(long long)k * total + idx];
    const int r = (int)(idx / N), c = (int)(idx % N);
    double* o = out + (long long)r * ldo + c;
    *o = (beta == 0.0) ? s : s + beta * (*o);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;

bool get_encode() {
  if (g_encode) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  g_encode = (EncodeTiledFn)fn;
  return true;
}

// 2-D map over a rows x ld operand part, boxes of 128 rows x 128 bytes, 128B swizzle
bool make_map(CUtensorMap* m, void* base, long long rows, long long ld, int prec) {
  const int es = tc_elem_bytes(prec);
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
  cuuint32_t box[2] = {(cuuint32_t)(KROW / es), (cuuint32_t)BM};
  cuuint32_t el[2] = {1, 1};
  const CUtensorMapDataType dt = (prec == TC_TF32X3) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  return g_encode(m, dt, 2, base, dims, strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int tc_gemm(Exec& ex, const TcGemm& g) {
  if (g.M <= 0 || g.N <= 0) return MOLGW_OK;
  const int ke = tc_kblock(g.prec);
  const int ns = tc_slices(g.prec);
  if (g.K <= 0 || g.K % ke || g.A.ld % ke || g.B.ld % ke || g.K > g.A.ld || g.K > g.B.ld) return MOLGW_E_ARG;
  if (ns == 3 && (!g.A.lo2 || !g.B.lo2)) return MOLGW_E_ARG;
  if (!get_encode()) return MOLGW_E_CUDA;
  CUtensorMap ma[3], mb[3];
  void* pa[3] = {g.A.hi, g.A.lo, ns == 3 ? g.A.lo2 : g.A.lo};
  void* pb[3] = {g.B.hi, g.B.lo, ns == 3 ? g.B.lo2 : g.B.lo};
  for (int k = 0; k < 3; ++k)
    if (!make_map(&ma[k], pa[k], g.A.rows, g.A.ld, g.prec) || !make_map(&mb[k], pb[k], g.B.rows, g.B.ld, g.prec))
      return MOLGW_E_ARG;
  KParams p;
  p.M = g.M; p.N = g.N;
  p.nkb = g.K / ke;
  int ks = std::max(1, std::min(g.ksplit, p.nkb));
  if (g.epi.mode != TC_EPI_F32_PARTIAL) ks = 1;
  p.kchunk = ceil_div(p.nkb, ks);
  p.ksplit = ceil_div(p.nkb, p.kchunk);
  p.batch = std::max(1, g.batch);
  p.lower_only = g.lower_only ? 1 : 0;
  p.a_batch_rows = g.a_batch_rows; p.b_batch_rows = g.b_batch_rows; p.out_batch_rows = g.out_batch_rows;
  p.epi = g.epi;
  p.status = ex.status;
  dim3 grid(ceil_div(g.N, BN), ceil_div(g.M, BM), p.batch * p.ksplit);
  KScope ks_(ex, MOLGW_K_GEMM_TC, 1);
  if (g.prec == TC_BF16X3) {
    cudaFuncSetAttribute(tc_gemm_kernel<TC_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, Ring<2>::SMEM);
    tc_gemm_kernel<TC_BF16X3><<<grid, 256, Ring<2>::SMEM, ex.st>>>(ma[0], ma[1], ma[2], mb[0], mb[1], mb[2], p);
  } else if (g.prec == TC_TF32X3) {
    cudaFuncSetAttribute(tc_gemm_kernel<TC_TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, Ring<2>::SMEM);
    tc_gemm_kernel<TC_TF32X3><<<grid, 256, Ring<2>::SMEM, ex.st>>>(ma[0], ma[1], ma[2], mb[0], mb[1], mb[2], p);
  } else {
    cudaFuncSetAttribute(tc_gemm_kernel<TC_BF16X6>, cudaFuncAttributeMaxDynamicSharedMemorySize, Ring<3>::SMEM);
    tc_gemm_kernel<TC_BF16X6><<<grid, 256, Ring<3>::SMEM, ex.st>>>(ma[0], ma[1], ma[2], mb[0], mb[1], mb[2], p);
  }
  return MOLGW_OK;
}

int tc_ksplit_of(int nkb, int ks) {
  ks = std::max(1, std::min(ks, nkb));
  const int chunk = ceil_div(nkb, ks);
  return ceil_div(nkb, chunk);
}

void tc_split(Exec& ex, int prec, const double* src, long long rows, long long cols, long long sr, long long sk,
              const double* row_scale, TcMat dst) {
  dim3 grid(ceil_div(dst.ld, 32), ceil_div(rows, 32));
  KScope ks(ex, MOLGW_K_MISC);
  if (prec == TC_BF16X3)
    k_split<TC_BF16X3><<<grid, dim3(32, 8), 0, ex.st>>>(src, rows, cols, sr, sk, row_scale, dst);
  else if (prec == TC_TF32X3)
    k_split<TC_TF32X3><<<grid, dim3(32, 8), 0, ex.st>>>(src, rows, cols, sr, sk, row_scale, dst);
  else
    k_split<TC_BF16X6><<<grid, dim3(32, 8), 0, ex.st>>>(src, rows, cols, sr, sk, row_scale, dst);
}

void tc_reduce_partials(Exec& ex, const float* part, int ksplit, int M, int N, double* out, long long ldo, double beta) {
  const long long total = (long long)M * N;
  KScope ks(ex, MOLGW_K_MISC);
  k_reduce_partials<<<(int)std::min<long long>(ceil_div(total, 256), 152LL * 8), 256, 0, ex.st>>>(part, ksplit, M, N,
                                                                                                    out, ldo, beta);
}

}  // namespace molgw
