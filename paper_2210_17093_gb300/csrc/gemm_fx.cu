// Fixed-point split GEMM (fx.cuh) on tcgen05 for sm_103a.
//
// Persistent CTAs (one per SM), each taking 128 x BN output tiles of one K group (<= 1024
// elements) in turn; 12 warps:
//   warp 0   TMA producer: the NS BF16 digit planes of a 128-row A box and a
//            BN-row B box per K block into a shared-memory ring;
//   warp 1   one thread issues tcgen05.mma (kind::f16, M=128, N=BN, K=16): per K
//            step the products of digit planes (a, b) with a + b = l accumulate
//            into level accumulator l (NS per buffer); after each chunk the
//            buffer is committed to the epilogue and the other buffer is used;
//   warp 2   allocates / frees the 512 TMEM columns (2 buffers x NS levels x BN);
//   warps 4-11 the epilogue: for each chunk, tcgen05.ld of the levels of its 32
//            lanes x BN/2 columns, conversion to integers (exact) and accumulation
//            of sum_l 2^(-8l) L_l in 64-bit integers (two words for NS = 7); after
//            the last chunk the words are joined in one 64-bit integer, rounded once
//            to float64 and scaled by u_a u_b (powers of two).
// Configurations:
//   NS = 4: K block 64 elements (128-byte swizzle), BN = 64, 256-element chunks,
//           2 stages of 96 KB;
//   NS = 7: K block 32 elements (64-byte swizzle), BN = 32, 128-element chunks,
//           3 stages of 70 KB.
// Every wait is bounded; a timeout latches MOLGW_E_TIMEOUT, raises a shared abort
// flag that ends the other roles' waits, and the CTA still frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include "fx.cuh"

namespace molgw {

namespace {

constexpr int BM = 128;
constexpr int TMEM_COLS = 512;
constexpr int NT = 384;
constexpr int EPI_THREADS = 256;
constexpr long long SPIN_LIMIT = 1LL << 26;

template <int NS> struct FxT;
template <> struct FxT<4> {
  static constexpr int KE = 64, BN = 64, CHUNK = 256, STAGES = 2, LAYOUT = 2, SBO = 1024;
};
template <> struct FxT<7> {
  static constexpr int KE = 32, BN = 32, CHUNK = 128, STAGES = 3, LAYOUT = 4, SBO = 512;
};
template <int NS> struct FxK : FxT<NS> {
  using B = FxT<NS>;
  static constexpr int ROWB = B::KE * 2;                 // bytes per K row of a box
  static constexpr int TA = BM * ROWB, TB = B::BN * ROWB;
  static constexpr int STAGE = NS * (TA + TB);
  static constexpr int SMEM = B::STAGES * STAGE + 1024;
  static constexpr int KSTEPS = B::KE / 16;
  static constexpr int KB_CHUNK = B::CHUNK / B::KE;
  static constexpr int KB_GROUP = kFxGroup / B::KE;
  static constexpr int LEVEL_COLS = NS * B::BN;          // TMEM columns of one buffer
  static constexpr int CPT = B::BN / 2;                  // epilogue columns per thread
  static_assert(2 * LEVEL_COLS <= TMEM_COLS, "two accumulator buffers must fit in TMEM");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t cnt) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// bounded wait on a phase parity; gives up early when another role raised *abort
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort) {
  const uint32_t a = smem_u32(b);
  for (long long it = 0; it < SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255 && *abort) return false;
  }
  return false;
}
__device__ __forceinline__ void fail(int* status, volatile int* abort) {
  set_status(status, MOLGW_E_TIMEOUT);
  *abort = 1;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// K-major operand with a LAYOUT swizzle (2: 128-byte, 4: 64-byte), 8-row groups SBO bytes apart
template <int LAYOUT, int SBO>
__device__ __forceinline__ uint64_t sdesc(const void* p) {
  const uint32_t a = smem_u32(p);
  uint64_t d = (uint64_t)((a & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(SBO >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)LAYOUT << 61;
  return d;
}
__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

struct FxMaps {
  CUtensorMap a[kFxMaxSlices], b[kFxMaxSlices];
};

struct FxParams {
  int M, N, nkb, kb0;                 // K blocks (of the configuration's KE) in the range, first one
  int nz;                             // K groups (split-K partials)
  const double* ua;
  int a_ngroups;
  const double* ub;
  int b_ngroups;
  double* out;
  long long out_ld, split_stride;
  int col_major, accumulate, lower_only;
  double alpha;
  const double* diag;
  int* status;
};

template <int NS>
__global__ void __launch_bounds__(NT, 1) fx_gemm_kernel(const __grid_constant__ FxMaps maps, FxParams p) {
  using C = FxK<NS>;
  constexpr int BN = C::BN, STAGES = C::STAGES;
  // Persistent: CTA b takes tiles b, b + gridDim.x, ... of the (N/BN) x (M/BM) x (K groups)
  // grid, N fastest (neighbouring CTAs share A's rows).  Every role walks the same tile
  // sequence; the stage ring and the two TMEM buffers run on counters kept across tiles, so
  // the epilogue of one tile overlaps the next tile's copies and MMAs.
  const int ntx = (p.N + BN - 1) / BN, nty = (p.M + BM - 1) / BM;
  const long long ntiles = (long long)ntx * nty * p.nz;
  auto tile_at = [&](long long t, int& n0, int& m0, int& gz) {
    n0 = (int)(t % ntx) * BN;
    m0 = (int)((t / ntx) % nty) * BM;
    gz = (int)(t / ((long long)ntx * nty));
  };
  // only strictly-upper 64-blocks are skipped
  auto skip = [&](int n0, int m0) { return p.lower_only && n0 / 64 > (m0 + BM - 1) / 64; };
  auto k_blocks = [&](int gz) { return min(p.nkb - gz * C::KB_GROUP, C::KB_GROUP); };

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[STAGES], empty[STAGES], accf[2], acce[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], EPI_THREADS);
    }
    mbar_init(&drain, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base;
  volatile int* abort = &abort_flag;

  if (warp == 0 && lane == 0) {
    int issued = 0;                               // K blocks copied, over all tiles
    bool ok = true;
    for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int n0, m0, gz;
      tile_at(t, n0, m0, gz);
      if (skip(n0, m0)) continue;
      const int kbl0 = gz * C::KB_GROUP, nk = k_blocks(gz);
      for (int i = 0; i < nk; ++i) {
        const int gi = issued, s = gi % STAGES;
        if (gi >= STAGES && !mbar_wait(&empty[s], ((gi / STAGES) + 1) & 1, abort)) {
          fail(p.status, abort);
          ok = false;
          break;
        }
        uint8_t* st = smem + s * C::STAGE;
        mbar_expect_tx(&full[s], C::STAGE);
        const int x = (p.kb0 + kbl0 + i) * C::KE;
#pragma unroll
        for (int sl = 0; sl < NS; ++sl) {
          tma_load_2d(st + sl * C::TA, &maps.a[sl], &full[s], x, m0);
          tma_load_2d(st + NS * C::TA + sl * C::TB, &maps.b[sl], &full[s], x, n0);
        }
        issued = gi + 1;
      }
    }
    // copies in flight (on an error path) land before the CTA leaves
    for (int i = (issued > STAGES ? issued - STAGES : 0); i < issued; ++i) {
      const uint32_t a = smem_u32(&full[i % STAGES]);
      for (long long it = 0; it < SPIN_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}"
            : "=r"(done)
            : "r"(a), "r"((uint32_t)((i / STAGES) & 1))
            : "memory");
        if (done) break;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // D F32 (bit 4); A, B BF16 (1 at bits 7 and 10); K-major; N>>3 at bit 17; M>>4 at bit 24
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    int i = 0;                                    // K blocks consumed, over all tiles
    int c = 0;                                    // chunks, over all tiles (TMEM buffer c & 1)
    bool ok = true;
    for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int n0, m0, gz;
      tile_at(t, n0, m0, gz);
      if (skip(n0, m0)) continue;
      const int nk = k_blocks(gz);
      const int nchunk = (nk + C::KB_CHUNK - 1) / C::KB_CHUNK;
      for (int cc = 0; cc < nchunk && ok; ++cc, ++c) {
        const int buf = c & 1;
        if (c >= 2 && !mbar_wait(&acce[buf], ((c >> 1) + 1) & 1, abort)) {
          fail(p.status, abort);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int kbn = min(C::KB_CHUNK, nk - cc * C::KB_CHUNK);
        for (int kb = 0; kb < kbn; ++kb, ++i) {
          const int s = i % STAGES;
          if (!mbar_wait(&full[s], (i / STAGES) & 1, abort)) {
            fail(p.status, abort);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          uint8_t* st = smem + s * C::STAGE;
#pragma unroll
          for (int kk = 0; kk < C::KSTEPS; ++kk) {   // 32 bytes of K per step
            const uint64_t o = 2 * kk;                // +32 B in the 16-byte-encoded address field
#pragma unroll
            for (int l = 0; l < NS; ++l)
#pragma unroll
              for (int a = 0; a <= l; ++a) {
                const int b = l - a;
                const uint64_t ad = sdesc<C::LAYOUT, C::SBO>(st + a * C::TA) + o;
                const uint64_t bd = sdesc<C::LAYOUT, C::SBO>(st + NS * C::TA + b * C::TB) + o;
                const uint32_t dt = tbase + (uint32_t)(buf * C::LEVEL_COLS + l * BN);
                mma_bf16(dt, ad, bd, idesc, (kb > 0 || kk > 0 || a > 0) ? 1u : 0u);
              }
          }
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&accf[buf]);
      }
    }
    if (!ok && i > 0) {
      // error path: the MMAs already issued finish before TMEM is released (bounded
      // wait that the abort flag does not cut short)
      mma_commit(&drain);
      const uint32_t a = smem_u32(&drain);
      for (long long it = 0; it < SPIN_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}"
            : "=r"(done)
            : "r"(a), "r"(0u)
            : "memory");
        if (done) break;
      }
    }
  } else if (warp >= 4) {
    const int q = warp & 3, h = (warp - 4) >> 2;            // TMEM lane quarter, column half
    const int lrow = 32 * q + lane;
    constexpr int CPT = C::CPT;
    constexpr int NL = (NS == 7) ? CPT : 1;
    int c = 0;                                              // chunks, over all tiles
    bool ok = true;
    for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int n0, m0, gz;
      tile_at(t, n0, m0, gz);
      if (skip(n0, m0)) continue;
      const int row = m0 + lrow;
      const int nk = k_blocks(gz);
      const int nchunk = (nk + C::KB_CHUNK - 1) / C::KB_CHUNK;
      const int group = (p.kb0 + gz * C::KB_GROUP) / C::KB_GROUP;   // scale group index of the operands
      long long Vh[CPT], Vl[NL];                            // Vl: levels 4.. (NS = 7 only)
#pragma unroll
      for (int j = 0; j < CPT; ++j) Vh[j] = 0;
#pragma unroll
      for (int j = 0; j < NL; ++j) Vl[j] = 0;
      for (int cc = 0; cc < nchunk; ++cc, ++c) {
        const int buf = c & 1;
        const bool got = mbar_wait(&accf[buf], (c >> 1) & 1, abort);
        if (!got) fail(p.status, abort);
        ok = __all_sync(0xffffffffu, got);       // the TMEM loads below are warp-collective
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int cb = 0; cb < CPT / 8; ++cb) {
          uint32_t r[NS][8];
#pragma unroll
          for (int l = 0; l < NS; ++l)
            tmem_ld8(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * C::LEVEL_COLS + l * BN + h * CPT + cb * 8),
                     r[l]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            // every level sum is an integer below 2^24: the conversions are exact
            long long L[NS];
#pragma unroll
            for (int l = 0; l < NS; ++l) L[l] = __float2int_rn(__uint_as_float(r[l][jj]));
            Vh[cb * 8 + jj] += (L[0] << 24) + (L[1] << 16) + (L[2] << 8) + L[3];
            if constexpr (NS == 7) Vl[cb * 8 + jj] += (L[4] << 16) + (L[5] << 8) + L[6];
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&acce[buf]);
      }
      if (ok && row < p.M) {
        // value = 2^-24 Vh u_a u_b (4 digits) or 2^-48 (2^24 Vh + Vl) u_a u_b (7 digits), formed
        // in integers as T = 2^14 Vh + floor(Vl / 2^10) = floor((2^24 Vh + Vl) / 2^10) (below
        // 2^63: |Vh| < 2^49 for a 1024-element group) and rounded once to float64; the scales
        // are powers of two (and alpha folded into u_a), so the float64 work per element is
        // a conversion, a multiply and the fused multiply-add into the output
        const double ua = p.ua[(long long)row * p.a_ngroups + group] * (NS == 7 ? 0x1p-38 : 0x1p-24);
        const double uaa = p.accumulate ? ua * p.alpha : ua;
        double* out = p.out + (long long)gz * p.split_stride;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const int col = n0 + h * CPT + j;
          if (col < p.N && !(p.lower_only && row / 64 < col / 64)) {
            long long T = Vh[j];
            if constexpr (NS == 7) T = (Vh[j] << 14) + (Vl[j] >> 10);
            const double v = (double)T;
            const double sc = uaa * p.ub[(long long)col * p.b_ngroups + group];
            double* o = p.col_major ? out + (long long)col * p.out_ld + row : out + (long long)row * p.out_ld + col;
            if (p.accumulate) {
              *o = fma(v, sc, *o);
            } else {
              double w = v * sc;
              if (p.diag && row == col) w += p.diag[row] * p.diag[row];
              *o = w;
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
  }
}

__global__ void k_fx_reduce_rm(const double* __restrict__ part, int ns, long long ss, int M, int N, double* out,
                               long long ldo, double beta) {
  const long long total = (long long)M * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / N), c = (int)(idx % N);
    double s = 0.0;
    for (int k = 0; k < ns; ++k) s += part[k * ss + idx];
    double* o = out + (long long)r * ldo + c;
    *o = (beta == 0.0) ? s : s + beta * (*o);
  }
}

__global__ void k_fx_reduce_cm(const double* __restrict__ part, int ns, long long ss, int M, int N, double* out,
                               long long ldo, double beta) {
  const long long total = (long long)M * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx % M), c = (int)(idx / M);
    double s = 0.0;
    for (int k = 0; k < ns; ++k) s += part[k * ss + idx];
    double* o = out + (long long)r * ldo + c;
    *o = (beta == 0.0) ? s : s + beta * (*o);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode_fx = nullptr;

bool get_encode_fx() {
  if (g_encode_fx) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  g_encode_fx = (EncodeTiledFn)fn;
  return true;
}

// BF16 digit-plane map: boxes of box_rows rows x ke elements, swizzle of ke * 2 bytes
bool make_map_fx(CUtensorMap* m, void* base, long long rows, long long ld, int box_rows, int ke) {
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)ke, (cuuint32_t)box_rows};
  cuuint32_t el[2] = {1, 1};
  const CUtensorMapSwizzle sw = (ke == 64) ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  return g_encode_fx(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NS>
int fx_launch(Exec& ex, const FxGemm& g) {
  using C = FxK<NS>;
  FxMaps maps;
  for (int i = 0; i < NS; ++i)
    if (!make_map_fx(&maps.a[i], g.A.s[i], g.A.rows, g.A.ld, BM, C::KE) ||
        !make_map_fx(&maps.b[i], g.B.s[i], g.B.rows, g.B.ld, C::BN, C::KE))
      return MOLGW_E_ARG;
  FxParams p;
  p.M = g.M; p.N = g.N;
  p.nkb = g.K / C::KE;
  p.kb0 = g.k0 / C::KE;
  p.ua = g.A.u; p.a_ngroups = g.A.ngroups;
  p.ub = g.B.u; p.b_ngroups = g.B.ngroups;
  p.out = g.out; p.out_ld = g.out_ld; p.split_stride = g.split_stride;
  p.col_major = g.col_major ? 1 : 0;
  p.accumulate = g.accumulate ? 1 : 0;
  p.lower_only = g.lower_only ? 1 : 0;
  p.alpha = g.alpha;
  p.diag = g.accumulate ? nullptr : g.diag;
  p.status = ex.status;
  p.nz = fx_nsplit(g.K);
  // persistent CTAs, one per SM (the stage ring and TMEM hold one per SM), at most one per tile
  const long long tiles = (long long)ceil_div(g.N, C::BN) * ceil_div(g.M, BM) * p.nz;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, std::max(sms, 1)));
  KScope ks(ex, g.kclass, 1);
  cudaFuncSetAttribute(fx_gemm_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  fx_gemm_kernel<NS><<<grid, NT, C::SMEM, ex.st>>>(maps, p);
  return MOLGW_OK;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

size_t fx_mat_bytes(long long rows, long long ld, int ns) {
  return ns * align256((size_t)rows * ld * 2) + align256((size_t)rows * fx_groups(ld) * sizeof(double));
}

FxMat fx_mat_carve(void* base, long long rows, long long ld, int ns) {
  FxMat m;
  m.rows = rows;
  m.ld = ld;
  m.ngroups = fx_groups(ld);
  m.ns = ns;
  char* p = (char*)base;
  for (int i = 0; i < ns; ++i) {
    m.s[i] = p;
    p += align256((size_t)rows * ld * 2);
  }
  m.u = (double*)p;
  return m;
}

FxMat fx_rows(const FxMat& m, long long r0, long long rows) {
  FxMat v = m;
  for (int i = 0; i < m.ns; ++i) v.s[i] = (char*)m.s[i] + r0 * m.ld * 2;
  v.u = m.u + r0 * m.ngroups;
  v.rows = rows;
  return v;
}

int fx_gemm(Exec& ex, const FxGemm& g) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return MOLGW_OK;
  if (g.A.ns != g.B.ns || (g.A.ns != 4 && g.A.ns != 7)) return MOLGW_E_ARG;
  if (g.K % kFxKBlock || g.k0 % kFxGroup || g.A.ld % kFxKBlock || g.B.ld % kFxKBlock || g.k0 + g.K > g.A.ld ||
      g.k0 + g.K > g.B.ld || g.M > g.A.rows || g.N > g.B.rows)
    return MOLGW_E_ARG;
  if (g.accumulate && fx_nsplit(g.K) != 1) return MOLGW_E_ARG;
  if (!get_encode_fx()) return MOLGW_E_CUDA;
  return g.A.ns == 7 ? fx_launch<7>(ex, g) : fx_launch<4>(ex, g);
}

void fx_split(Exec& ex, const double* src, long long rows, long long cols, long long sr, long long sk,
              const double* row_scale, FxMat dst, int kclass) {
  if (sk == 1 && sr != 1) {
    if (rows <= 0) return;
    KScope ks(ex, kclass, 1);
    const long long warps = rows * dst.ngroups;
    const int blocks = ceil_div(warps, 8);
    if (dst.ns == 7)
      k_fx_rows<7><<<blocks, 256, 0, ex.st>>>(src, rows, cols, sr, row_scale, dst);
    else
      k_fx_rows<4><<<blocks, 256, 0, ex.st>>>(src, rows, cols, sr, row_scale, dst);
    return;
  }
  FxStrided f{src, sr, sk, rows, cols, row_scale};
  fx_slice(ex, f, rows, dst, kclass);
}

void fx_reduce_rm(Exec& ex, const double* part, int ns, long long split_stride, int M, int N, double* out,
                  long long ldo, double beta) {
  const long long total = (long long)M * N;
  KScope ks(ex, MOLGW_K_MISC);
  k_fx_reduce_rm<<<(int)std::min<long long>(ceil_div(total, 256), 152LL * 8), 256, 0, ex.st>>>(
      part, ns, split_stride, M, N, out, ldo, beta);
}

void fx_reduce_cm(Exec& ex, const double* part, int ns, long long split_stride, int M, int N, double* out,
                  long long ldo, double beta) {
  const long long total = (long long)M * N;
  KScope ks(ex, MOLGW_K_MISC);
  k_fx_reduce_cm<<<(int)std::min<long long>(ceil_div(total, 256), 152LL * 8), 256, 0, ex.st>>>(
      part, ns, split_stride, M, N, out, ldo, beta);
}

}  // namespace molgw
