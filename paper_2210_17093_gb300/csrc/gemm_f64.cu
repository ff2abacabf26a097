// Float64 GEMM on the CUDA cores (DFMA) for the plain-FP64 path.
//
// On GB300 the FP64 pipe delivers about 2 DFMA per clock per SM (measured
// 1.2 TFLOP/s over 152 SMs), so a 64x64x16 shared-memory tile with a 4x4
// register block per thread needs ~0.25 byte/FMA of L2 traffic and is bound by
// the FP64 pipe, not by memory.  The kernel takes arbitrary element strides so
// that one routine serves every contraction of the pass (row- or column-major
// operands, batched over an auxiliary index, transposed views).
#include "common.cuh"

namespace molgw {

namespace {

constexpr int TK = 16;
constexpr int TM = 64, TN = 64;   // tile of the lower_only bookkeeping (64x64 tiles)

struct GemmParams {
  int M, N, K, batch, ksplit, kchunk;
  const double* A; long long sa_m, sa_k, sa_b;
  const double* B; long long sb_k, sb_n, sb_b;
  double* C; long long sc_m, sc_n, sc_b;
  double alpha, beta;
  int lower_only;
  double* work;
};

// BM x BN output tile per CTA, (BM/4) x (BN/4) threads, 4x4 outputs per thread
// (rows ty + (BM/4) i, columns tx + (BN/4) j).
template <int BM, int BN>
__global__ void __launch_bounds__((BM / 4) * (BN / 4)) gemm_f64_kernel(GemmParams p) {
  constexpr int TX = BN / 4, TY = BM / 4, NTH = TX * TY;
  const int bn = blockIdx.x, bm = blockIdx.y;
  if (p.lower_only && bm < bn) return;   // lower_only is used with BM = BN = 64 only
  const int z = blockIdx.z;
  const int b = z % p.batch, kz = z / p.batch;
  const int k_begin = kz * p.kchunk;
  const int k_end = min(p.K, k_begin + p.kchunk);

  __shared__ double As[TK][BM + 1];
  __shared__ double Bs[TK][BN + 1];

  const int t = threadIdx.x;
  const int tx = t % TX, ty = t / TX;
  const int m0 = bm * BM, n0 = bn * BN;
  const double* A = p.A + (long long)b * p.sa_b;
  const double* B = p.B + (long long)b * p.sb_b;
  const bool a_kfast = (p.sa_k == 1);
  const bool b_nfast = (p.sb_n == 1);

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = k_begin; k0 < k_end; k0 += TK) {
    for (int e = t; e < BM * TK; e += NTH) {
      int m, k;
      if (a_kfast) { k = e % TK; m = e / TK; }
      else { m = e % BM; k = e / BM; }
      const int gm = m0 + m, gk = k0 + k;
      As[k][m] = (gm < p.M && gk < k_end) ? A[(long long)gm * p.sa_m + (long long)gk * p.sa_k] : 0.0;
    }
    for (int e = t; e < BN * TK; e += NTH) {
      int n, k;
      if (b_nfast) { n = e % BN; k = e / BN; }
      else { k = e % TK; n = e / TK; }
      const int gn = n0 + n, gk = k0 + k;
      Bs[k][n] = (gn < p.N && gk < k_end) ? B[(long long)gk * p.sb_k + (long long)gn * p.sb_n] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + TY * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[k][tx + TX * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }

  if (p.ksplit > 1) {
    double* W = p.work + ((long long)kz * p.batch + b) * (long long)p.M * p.N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + ty + TY * i;
      if (gm >= p.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gn = n0 + tx + TX * j;
        if (gn < p.N) W[(long long)gm * p.N + gn] = acc[i][j];
      }
    }
    return;
  }
  double* C = p.C + (long long)b * p.sc_b;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + TY * i;
    if (gm >= p.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + TX * j;
      if (gn >= p.N) continue;
      double* c = C + (long long)gm * p.sc_m + (long long)gn * p.sc_n;
      const double v = p.alpha * acc[i][j];
      *c = (p.beta == 0.0) ? v : fma(p.beta, *c, v);
    }
  }
}

// C = alpha * sum_kz work[kz] + beta * C, summed in kz order.
__global__ void gemm_splitk_reduce(GemmParams p) {
  const long long mn = (long long)p.M * p.N;
  const long long total = mn * p.batch;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(idx / mn);
    const long long r = idx % mn;
    const int gm = (int)(r / p.N), gn = (int)(r % p.N);
    if (p.lower_only && (gm / TM) < (gn / TN)) continue;
    double s = 0.0;
    for (int kz = 0; kz < p.ksplit; ++kz) s += p.work[((long long)kz * p.batch + b) * mn + r];
    double* c = p.C + (long long)b * p.sc_b + (long long)gm * p.sc_m + (long long)gn * p.sc_n;
    const double v = p.alpha * s;
    *c = (p.beta == 0.0) ? v : fma(p.beta, *c, v);
  }
}

}  // namespace

// Output tile side with the least padding (64, 48, 40 or 32).
int pick_tile(int M) {
  const int cand[4] = {64, 48, 40, 32};
  int best = 64;
  double best_eff = 0.0;
  for (int c : cand) {
    const double eff = (double)M / (ceil_div(M, c) * c);
    if (eff > best_eff + 0.02) { best = c; best_eff = eff; }
  }
  return best;
}

int gemm_f64_pick_split(int M, int N, int K, int batch, size_t work_cap_doubles) {
  const long long tiles = (long long)ceil_div(M, TM) * ceil_div(N, TN) * batch;
  const long long target = 152LL * 4;
  if (tiles >= target || K < 512) return 1;
  long long ks = (target + tiles - 1) / tiles;
  ks = std::min<long long>(ks, K / 256);
  const long long per = (long long)M * N * batch;
  if (per > 0) ks = std::min<long long>(ks, (long long)(work_cap_doubles / per));
  return (int)std::max<long long>(1, std::min<long long>(ks, 64));
}

namespace {

long long bucket(long long x) {
  // the smallest of {4, 5, 6, 7} x 2^k (k >= 0) that is >= x
  if (x <= 4) return x;
  long long b = 4;
  while (b * 2 < x) b *= 2;
  for (long long f = 4; f <= 8; ++f)
    if (b / 4 * f >= x) return b / 4 * f;
  return b * 2;
}

void launch_side(Exec& ex, const GemmParams& p, int side, int kclass, int M, int N, int batch) {
  dim3 grid(ceil_div(N, side), ceil_div(M, side), batch * p.ksplit);
  KScope ks(ex, kclass, p.ksplit > 1 ? 2 : 1);
  switch (side) {
    case 48: gemm_f64_kernel<48, 48><<<grid, 144, 0, ex.st>>>(p); break;
    case 40: gemm_f64_kernel<40, 40><<<grid, 100, 0, ex.st>>>(p); break;
    case 32: gemm_f64_kernel<32, 32><<<grid, 64, 0, ex.st>>>(p); break;
    default: gemm_f64_kernel<64, 64><<<grid, 256, 0, ex.st>>>(p); break;
  }
  if (p.ksplit > 1) {
    const long long total = (long long)M * N * batch;
    const int blocks = (int)std::min<long long>(ceil_div(total, 256), 152LL * 16);
    gemm_splitk_reduce<<<blocks, 256, 0, ex.st>>>(p);
  }
}

// Time every tile side on the shape of p with the output redirected to the tuner's
// scratch (beta = 0, the same majorness); returns the fastest side, or 0.
int tune_side(Exec& ex, const GemmParams& p0, int M, int N, int batch) {
  GemmTuner& t = *ex.tuner;
  const size_t need = (size_t)M * N * batch;
  if (need > ((size_t)64 << 20)) return 0;
  if (need > t.scratch_cap) {
    cudaStreamSynchronize(ex.st);
    if (t.scratch) cudaFree(t.scratch);
    t.scratch = nullptr;
    t.scratch_cap = 0;
    if (cudaMalloc(&t.scratch, need * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return 0; }
    t.scratch_cap = need;
  }
  if (!t.e0) { cudaEventCreate(&t.e0); cudaEventCreate(&t.e1); }
  GemmParams p = p0;
  p.C = t.scratch;
  p.beta = 0.0;
  if (p0.sc_m == 1) { p.sc_m = 1; p.sc_n = M; } else { p.sc_m = N; p.sc_n = 1; }
  p.sc_b = (long long)M * N;
  Exec quiet = ex;
  quiet.timer = nullptr;
  int best = 0;
  float best_ms = 0.0f;
  for (int side : {64, 48, 40, 32}) {
    cudaEventRecord(t.e0, ex.st);
    launch_side(quiet, p, side, MOLGW_K_MISC, M, N, batch);
    cudaEventRecord(t.e1, ex.st);
    if (cudaEventSynchronize(t.e1) != cudaSuccess) { cudaGetLastError(); return 0; }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, t.e0, t.e1);
    if (best == 0 || ms < best_ms) { best = side; best_ms = ms; }
  }
  ++t.tuned;
  return best;
}

}  // namespace

void gemm_f64(Exec& ex, const GemmF64& g) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  GemmParams p;
  p.M = g.M; p.N = g.N; p.K = g.K; p.batch = g.batch;
  p.ksplit = (g.ksplit > 1 && g.work) ? g.ksplit : 1;
  p.kchunk = ceil_div(std::max(g.K, 1), p.ksplit);
  p.kchunk = ceil_div(p.kchunk, TK) * TK;
  p.ksplit = std::max(1, ceil_div(std::max(g.K, 1), p.kchunk));
  p.A = g.A; p.sa_m = g.sa_m; p.sa_k = g.sa_k; p.sa_b = g.sa_b;
  p.B = g.B; p.sb_k = g.sb_k; p.sb_n = g.sb_n; p.sb_b = g.sb_b;
  p.C = g.C; p.sc_m = g.sc_m; p.sc_n = g.sc_n; p.sc_b = g.sc_b;
  p.alpha = g.alpha; p.beta = g.beta;
  p.lower_only = g.lower_only ? 1 : 0;
  p.work = g.work;
  // tile: 64x64 for lower_only (its tiles must align with the 64-blocked storage),
  // else the side that pads M and N least
  const int bm = g.lower_only ? 64 : pick_tile(g.M);
  const int bnn = g.lower_only ? 64 : pick_tile(g.N);
  int side = std::min(bm, bnn) == 64 ? 64 : std::max(std::min(bm, bnn), 32);
  if (ex.tuner && !g.lower_only) {
    const std::vector<long long> key = {bucket(g.M), bucket(g.N), bucket(g.K), g.batch, p.ksplit > 1,
                                        g.sa_m == 1, g.sa_k == 1, g.sb_k == 1, g.sb_n == 1, g.sc_m == 1};
    int found = 0;
    for (const auto& e : ex.tuner->best)
      if (e.first == key) { found = e.second; break; }
    if (!found && ex.tuner->active && !ex.capturing) {
      found = tune_side(ex, p, g.M, g.N, g.batch);
      if (found) ex.tuner->best.push_back({key, found});
    }
    if (found) side = found;
  }
  launch_side(ex, p, side, g.kclass, g.M, g.N, g.batch);
}

}  // namespace molgw
