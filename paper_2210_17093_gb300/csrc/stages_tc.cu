// Stages (a), (b), (d)+(e) on the split-precision tensor-core engine.
//
// (a) X_P = C^T L_P (batched over P, split output), B_P = X_P C (float64 output);
// (b) M = Xv Xv^T + D^2 with Xv = 2 D^1/2 B_ia^T, float64 epilogue, lower tiles;
// (d)+(e) for each block of m: w_m = B_m^T R (rows (m, p), columns s), whose
//     epilogue takes the float64 differences eps_p - eps_m -/+ Omega_s, forms
//     g = x / (x^2 + eta^2) and writes w and g*w as split operands laid out
//     [p][m*sp + s]; then S += (g w) w^T over K = (m, s) with split-K float32
//     partials reduced in a fixed order in float64.
// The eigensolvers (c), (f) and the back-transformation stay in float64.
#include "stages.cuh"
#include "tc.cuh"

namespace molgw {

namespace {

constexpr int kW = 64;                              // K elements per float32 chunk of w
constexpr long long kWpartFloats = 1LL << 28;       // float32 chunk partials of w: at most 1 GB

// Float32 K chunks of w = B_m^T R: one per kW elements of n_aux, fewer when the
// partials of one m would not fit in kWpartFloats.
int sigma_kw(int prec, int nb, int na, long long nov) {
  const int kb = tc_kblock(prec);
  const int nkw = (int)(tc_pad(na, prec) / kb);
  const long long fit = std::max<long long>(1, kWpartFloats / std::max<long long>((long long)nb * nov, 1));
  const int want = (int)std::min<long long>(ceil_div(nkw, std::max(1, kW / kb)), fit);
  return tc_ksplit_of(nkw, std::max(want, 1));
}

long long wpart_floats_for(int prec, int nb, int na, long long nov, int mb) {
  const long long per_m = (long long)sigma_kw(prec, nb, na, nov) * nb * nov;
  return std::min<long long>(std::max<long long>(per_m, (long long)mb * per_m), std::max(kWpartFloats, per_m));
}

TcMat carve(double*& base_bytes_as_double, long long rows, long long ld, int prec) {
  // carve the slices (each rows x ld elements) from a byte arena kept in doubles
  TcMat m;
  m.rows = rows;
  m.ld = ld;
  const long long bytes = rows * ld * tc_elem_bytes(prec);
  const long long words = (bytes + 255) / 256 * 32;   // 256-byte aligned, in doubles
  m.hi = base_bytes_as_double;
  base_bytes_as_double += words;
  m.lo = base_bytes_as_double;
  base_bytes_as_double += words;
  if (tc_slices(prec) == 3) {
    m.lo2 = base_bytes_as_double;
    base_bytes_as_double += words;
  }
  return m;
}

long long carve_doubles(long long rows, long long ld, int prec) {
  const long long bytes = rows * ld * tc_elem_bytes(prec);
  return tc_slices(prec) * ((bytes + 255) / 256 * 32);
}

// w = sum of the float32 chunk partials in float64; x = (eps_p - eps_m) -/+ Omega_s in
// float64; g = x / (x^2 + eta^2); w and g*w stored as split operands [p][mm*sp + s].
template <int PREC>
__global__ void k_sigma_combine(const float* __restrict__ part, int kw, long long rows, long long nov,
                                const double* __restrict__ eps, const double* __restrict__ omega, int nb, int no,
                                int m0, long long sp, double eta, TcMat W, TcMat P) {
  // every padded column sidx in [n_ov, sp) is written as zero: the operands are
  // carved from a lane arena that other molecules also use
  const long long total = rows * sp, ptotal = rows * nov;
  const double eta2 = eta * eta;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long row = idx / sp, sidx = idx % sp;
    const int mm = (int)(row / nb), pp = (int)(row % nb), m = m0 + mm;
    const long long o = (long long)pp * W.ld + (long long)mm * sp + sidx;
    if (sidx >= nov) {
      tc_store_split<PREC>(W, o, 0.0);
      tc_store_split<PREC>(P, o, 0.0);
      continue;
    }
    const long long pidx = row * nov + sidx;
    double w = 0.0;
    for (int k = 0; k < kw; ++k) w += (double)part[(long long)k * ptotal + pidx];
    const double x = (eps[pp] - eps[m]) + ((m < no) ? omega[sidx] : -omega[sidx]);
    const double g = x / (x * x + eta2);
    tc_store_split<PREC>(W, o, w);
    tc_store_split<PREC>(P, o, w * g);
  }
}

}  // namespace

size_t tc_ri_doubles(int prec, int nb, int na) {
  return (size_t)carve_doubles((long long)na * nb, tc_pad(nb, prec), prec);
}

size_t tc_orb_doubles(int prec, int nb, int na, long long nov, int mb) {
  const long long nbp = tc_pad(nb, prec), nap = tc_pad(na, prec), sp = tc_pad(nov, prec);
  size_t t = 0;
  t += carve_doubles(nb, nbp, prec);                 // C^T
  t += carve_doubles((long long)na * nb, nbp, prec); // X
  t += carve_doubles(nov, nap, prec);                // Xv
  t += carve_doubles(nov, nap, prec);                // R^T
  t += carve_doubles((long long)nb * nb, nap, prec); // B^T per m
  t += 2 * carve_doubles(nb, (long long)mb * sp, prec);   // w, g*w
  t += (wpart_floats_for(prec, nb, na, nov, mb) + 63) / 64 * 32;   // float32 chunk partials of w
  return t;
}

void tc_bufs_carve(TcBufs& t, int prec, int nb, int na, long long nov, int mb, double* base) {
  const long long nbp = tc_pad(nb, prec), nap = tc_pad(na, prec);
  t.prec = prec;
  t.mb = mb;
  t.sp = tc_pad(nov, prec);
  double* p = base;
  t.Ct = carve(p, nb, nbp, prec);
  t.X = carve(p, (long long)na * nb, nbp, prec);
  t.Xv = carve(p, nov, nap, prec);
  t.Rt = carve(p, nov, nap, prec);
  t.Bt = carve(p, (long long)nb * nb, nap, prec);
  t.W = carve(p, nb, (long long)mb * t.sp, prec);
  t.P = carve(p, nb, (long long)mb * t.sp, prec);
  t.wpart = reinterpret_cast<float*>(p);
  t.wpart_floats = wpart_floats_for(prec, nb, na, nov, mb);
}

void tc_ri_carve(TcBufs& t, int prec, int nb, int na, double* base) {
  double* p = base;
  t.prec = prec;
  t.L = carve(p, (long long)na * nb, tc_pad(nb, prec), prec);
}

// Split of L, once per set of RI factors: rows (P, nu), K = mu (L symmetric in mu nu).
void tc_split_ri(Exec& ex, MolBuf& m, TcBufs& t) {
  tc_split(ex, t.prec, m.L, (long long)m.na * m.nb, m.nb, m.nb, 1, nullptr, t.L);
}

int stage_ri_mo_transform_tc(Exec& ex, MolBuf& m, TcBufs& t) {
  const int nb = m.nb, na = m.na;
  const long long nbp = tc_pad(nb, t.prec);
  // C^T: element (p, mu) = C[mu][p]
  tc_split(ex, t.prec, m.C, nb, nb, 1, nb, nullptr, t.Ct);
  // X_P[q][nu] = sum_mu C[mu][q] L_P[nu][mu]
  TcGemm g1;
  g1.prec = t.prec;
  g1.M = nb; g1.N = nb; g1.K = (int)nbp;
  g1.A = t.Ct; g1.B = t.L;
  g1.batch = na; g1.a_batch_rows = 0; g1.b_batch_rows = nb; g1.out_batch_rows = nb;
  g1.epi.mode = TC_EPI_SPLIT;
  g1.epi.out_split = t.X;
  if (nbp > nb) {
    // the epilogue writes columns < nb; the K padding of X must read as zero
    const int es = tc_elem_bytes(t.prec);
    void* sl[3] = {t.X.hi, t.X.lo, t.X.lo2};
    for (int k = 0; k < tc_slices(t.prec); ++k)
      cudaMemset2DAsync((char*)sl[k] + (size_t)nb * es, (size_t)nbp * es, 0, (size_t)(nbp - nb) * es,
                        (size_t)na * nb, ex.st);
  }
  int r = tc_gemm(ex, g1);
  if (r) return r;
  // B[(P,q)][p] = sum_nu X[(P,q)][nu] C[nu][p]
  TcGemm g2;
  g2.prec = t.prec;
  g2.M = na * nb; g2.N = nb; g2.K = (int)nbp;
  g2.A = t.X; g2.B = t.Ct;
  g2.epi.mode = TC_EPI_F64;
  g2.epi.out_f64 = m.B;
  g2.epi.out_ld = nb;
  return tc_gemm(ex, g2);
}

int stage_rpa_build_tc(Exec& ex, MolBuf& m, TcBufs& t) {
  const int na = m.na;
  const long long nov = m.nov;
  gather_xv(ex, m);                                    // float64 Xv (column-major) and D
  tc_split(ex, t.prec, m.Xv, nov, na, 1, nov, nullptr, t.Xv);
  TcGemm g;
  g.prec = t.prec;
  g.M = (int)nov; g.N = (int)nov; g.K = (int)tc_pad(na, t.prec);
  g.A = t.Xv; g.B = t.Xv;
  g.lower_only = true;
  g.epi.mode = TC_EPI_RPA;
  g.epi.out_f64 = m.M;
  g.epi.out_ld = nov;
  g.epi.diag = m.D;
  return tc_gemm(ex, g);
}

int stage_sigma_tc(Exec& ex, MolBuf& m, TcBufs& t, Scratch& s, double eta) {
  const int nb = m.nb, na = m.na, no = m.no;
  const long long nov = m.nov, nn = (long long)nb * nb;
  const long long nap = tc_pad(na, t.prec);
  // R^T: element (s, P) = R[P][s];  B^T: element ((m, p), P) = B[P][m][p]
  tc_split(ex, t.prec, m.R, nov, na, 1, nov, nullptr, t.Rt);
  tc_split(ex, t.prec, m.B, nn, na, 1, nn, nullptr, t.Bt);
  const int es = tc_elem_bytes(t.prec);
  // w in K chunks of kW elements (float32 on the tensor cores), combined in float64
  const int kb = tc_kblock(t.prec);
  const int kw = sigma_kw(t.prec, nb, na, nov);
  const long long per_m = (long long)kw * nb * nov;   // floats of partials per m
  const int mstep = (int)std::max<long long>(1, std::min<long long>(t.mb, t.wpart_floats / std::max<long long>(per_m, 1)));
  for (int m0 = 0; m0 < nb; m0 += mstep) {
    const int cnt = std::min(mstep, nb - m0);
    TcGemm gw;
    gw.prec = t.prec;
    gw.M = cnt * nb; gw.N = (int)nov; gw.K = (int)nap;
    gw.A = t.Bt;
    gw.A.hi = (char*)t.Bt.hi + (long long)m0 * nb * nap * es;
    gw.A.lo = (char*)t.Bt.lo + (long long)m0 * nb * nap * es;
    gw.A.rows = (long long)cnt * nb;
    gw.B = t.Rt;
    gw.ksplit = kw;
    gw.epi.mode = TC_EPI_F32_PARTIAL;
    gw.epi.out_f32 = t.wpart;
    int r = tc_gemm(ex, gw);
    if (r) return r;
    {
      const long long total = (long long)cnt * nb * t.sp;
      const int blocks = (int)std::min<long long>(ceil_div(total, 256), 152LL * 16);
      KScope ks(ex, MOLGW_K_SIGMA);
      if (t.prec == TC_BF16X3)
        k_sigma_combine<TC_BF16X3><<<blocks, 256, 0, ex.st>>>(t.wpart, kw, (long long)cnt * nb, nov, m.eps, m.Om, nb,
                                                             no, m0, t.sp, eta, t.W, t.P);
      else if (t.prec == TC_TF32X3)
        k_sigma_combine<TC_TF32X3><<<blocks, 256, 0, ex.st>>>(t.wpart, kw, (long long)cnt * nb, nov, m.eps, m.Om, nb,
                                                             no, m0, t.sp, eta, t.W, t.P);
      else
        k_sigma_combine<TC_BF16X6><<<blocks, 256, 0, ex.st>>>(t.wpart, kw, (long long)cnt * nb, nov, m.eps, m.Om, nb,
                                                             no, m0, t.sp, eta, t.W, t.P);
    }
    TcGemm gs;
    gs.prec = t.prec;
    gs.M = nb; gs.N = nb; gs.K = (int)(cnt * t.sp);
    gs.A = t.P; gs.B = t.W;
    // split K = (m, s) into chunks of ~1024 products: the tensor cores accumulate
    // in float32, the partials are summed in float64
    int ks = std::max(1, gs.K / 1024);
    ks = std::min(ks, (int)(s.splitk_cap * 2 / std::max<long long>(nn, 1)));   // float partials in the double arena
    ks = tc_ksplit_of(gs.K / kb, std::max(ks, 1));
    gs.ksplit = ks;
    gs.epi.mode = TC_EPI_F32_PARTIAL;
    gs.epi.out_f32 = reinterpret_cast<float*>(s.splitk);
    r = tc_gemm(ex, gs);
    if (r) return r;
    tc_reduce_partials(ex, reinterpret_cast<float*>(s.splitk), ks, nb, nb, s.S, nb, m0 == 0 ? 0.0 : 1.0);
  }
  symmetrize(ex, s.S, nb, m.sigc);
  return MOLGW_OK;
}

}  // namespace molgw

// ---------------------------------------------------------------------------
// (d)+(e) on the fixed-point engine (fx.cuh): w = B_m^T R with exact chunk sums
// rounded once to float64; the float64 differences eps_p - eps_m -/+ Omega_s and
// g = x / (x^2 + eta^2) are formed while w and g*w are sliced; S += (g w) w^T over
// K = (m, s), one float64 partial per 1024-wide K group, summed in a fixed order.
// ---------------------------------------------------------------------------
namespace molgw {

namespace {

constexpr long long kFxBlockBytes = 1LL << 30;   // w and its slices per block of m

// 1/d by one Newton-Raphson step from a float32 seed: the relative error goes from
// ~2^-23 to ~2^-46, far below the 2^-32 (relative to a group's maximum) of the
// fixed-point digits made from it.  The range test runs on the float32 copy.  d > 0.
__device__ __forceinline__ double recip_newton(double d) {
  const float df = (float)d;
  if (!(df > 1e-30f && df < 1e30f)) return 1.0 / d;
  const double r = (double)__frcp_rn(df);
  return fma(r, fma(-d, r, 1.0), r);
}

constexpr int kSigRows = 4;   // rows p per block of k_fx_sigma_slices

// Digits of the two tiles held in shared memory (kSigRows rows each of one K group):
// warps 0..3 slice tile `tw` into W, warps 4..7 tile `tp` into P, one (row, group)
// scale each.
__device__ __forceinline__ void sigma_tiles_to_digits(const double* tw, const double* tp, int p0, int nb, int g,
                                                      long long k0, long long K, const FxMat& W, const FxMat& P) {
  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const int row = warp % kSigRows;
  const bool isP = warp >= kSigRows;
  const double* tile = (isP ? tp : tw) + row * kFxGroup;
  const FxMat& D = isP ? P : W;
  const int pr = p0 + row;
  if (pr >= nb) return;
  // max |x| on the bit patterns: for non-negative doubles the integer order is the value order
  long long mb = 0;
  for (int kk = lane; kk < kFxGroup; kk += 32) {
    const long long b = __double_as_longlong(tile[kk]) & 0x7fffffffffffffffLL;
    mb = b > mb ? b : mb;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const long long b = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = b > mb ? b : mb;
  }
  const double u = fx_unit(__longlong_as_double(mb));
  if (lane == 0) D.u[(long long)pr * D.ngroups + g] = u;
  const double scale24 = 0x1p24 / u;            // a power of two: exact
  for (int kk = lane; kk < kFxGroup && k0 + kk < K; kk += 32) {
    __nv_bfloat16 d[kFxSlices];
    fx_digits<kFxSlices>(tile[kk], scale24, d);
    const long long o = (long long)pr * D.ld + k0 + kk;
#pragma unroll
    for (int i = 0; i < kFxSlices; ++i) ((__nv_bfloat16*)D.s[i])[o] = d[i];
  }
}

// Slices of w and g*w for rows p0 .. p0+3 and one K group (K = mm*sp + s): w is
// the float64 sum of the group partials of the residue GEMM, x = (eps_p - eps_m)
// -/+ Omega_s in float64 and g = x / (x^2 + eta^2); each value is formed once,
// kept in shared memory for the (row, group) maxima, then sliced.
__global__ void __launch_bounds__(256) k_fx_sigma_slices(const double* __restrict__ wbuf, int nsplit,
                                                         long long split_stride, long long ldw, int sp, int nov,
                                                         int nb, int no, int m0, int cnt,
                                                         const double* __restrict__ eps,
                                                         const double* __restrict__ om, double eta2, FxMat W,
                                                         FxMat P) {
  extern __shared__ double sh[];
  double* tw = sh;                              // [kSigRows][kFxGroup]
  double* tp = sh + kSigRows * kFxGroup;
  const int p0 = blockIdx.x * kSigRows, g = blockIdx.y;
  const long long K = W.ld;
  const long long k0 = (long long)g * kFxGroup;
  const int t = threadIdx.x;
  const int r = t % kSigRows;
  const int p = p0 + r;
  for (int kk = t / kSigRows; kk < kFxGroup; kk += 256 / kSigRows) {
    const long long k = k0 + kk;
    double w = 0.0, gw = 0.0;
    if (p < nb && k < K) {
      const int mm = (int)(k / sp), s = (int)(k - (long long)mm * sp);
      if (mm < cnt && s < nov) {
        const long long o = (long long)s * ldw + (long long)mm * nb + p;
        w = wbuf[o];
        for (int j = 1; j < nsplit; ++j) w += wbuf[j * split_stride + o];
        const int m = m0 + mm;
        const double x = (eps[p] - eps[m]) + ((m < no) ? om[s] : -om[s]);   // float64 difference
        gw = w * (x * recip_newton(x * x + eta2));
      }
    }
    tw[r * kFxGroup + kk] = w;
    tp[r * kFxGroup + kk] = gw;
  }
  __syncthreads();
  sigma_tiles_to_digits(tw, tp, p0, nb, g, k0, K, W, P);
}

// qsMP2, Eq. (Sigma.c.MP2) with the frequency on row p, for rows p0 .. p0+3 and one
// K group (K = mm*sp + t, t = i*nv + a'): A = (p m|i a) from the group partials of
// the direct GEMM (layout of w above), X the exchange partner from its GEMMs'
// partials -- (m a|i p) at [mm][a'][i][p] for occupied m, (m i|a p) at [mm][i][a'][p]
// for empty m, p fastest as in w -- and x = (eps_p - eps_m) +/- D_t in float64.
// Tiles: A, and g(x) (2 A - X).
__global__ void __launch_bounds__(256) k_fx_mp2_slices(const double* __restrict__ wbuf,
                                                       const double* __restrict__ xbuf, int nsplit,
                                                       long long split_stride, long long ldw, int sp, int nov,
                                                       int nb, int no, int m0, int cnt,
                                                       const double* __restrict__ eps,
                                                       const double* __restrict__ dt, double eta2, FxMat W,
                                                       FxMat P) {
  extern __shared__ double sh[];
  double* tw = sh;
  double* tp = sh + kSigRows * kFxGroup;
  const int p0 = blockIdx.x * kSigRows, g = blockIdx.y;
  const long long K = W.ld;
  const long long k0 = (long long)g * kFxGroup;
  const int nv = nb - no;
  const int t = threadIdx.x;
  const int r = t % kSigRows;
  const int p = p0 + r;
  for (int kk = t / kSigRows; kk < kFxGroup; kk += 256 / kSigRows) {
    const long long k = k0 + kk;
    double a = 0.0, pv = 0.0;
    if (p < nb && k < K) {
      const int mm = (int)(k / sp), s = (int)(k - (long long)mm * sp);
      if (mm < cnt && s < nov) {
        const long long o = (long long)s * ldw + (long long)mm * nb + p;
        const int m = m0 + mm;
        const int i = s / nv, ap = s - i * nv;
        const long long ox = (long long)mm * nb * nov +
                             ((m < no) ? ((long long)ap * no + i) * nb + p : (long long)s * nb + p);
        a = wbuf[o];
        double x = xbuf[ox];
        for (int j = 1; j < nsplit; ++j) {
          a += wbuf[j * split_stride + o];
          x += xbuf[j * split_stride + ox];
        }
        const double d = (eps[p] - eps[m]) + ((m < no) ? dt[s] : -dt[s]);   // float64 difference
        pv = (2.0 * a - x) * (d * recip_newton(d * d + eta2));
      }
    }
    tw[r * kFxGroup + kk] = a;
    tp[r * kFxGroup + kk] = pv;
  }
  __syncthreads();
  sigma_tiles_to_digits(tw, tp, p0, nb, g, k0, K, W, P);
}
}  // namespace

namespace {

// element (r = P nb + p, k = mu) = T[P][mu][p] of T = L C (for B_P = C^T T_P, read
// transposed through the symmetry of B_P)
struct TSrc {
  const double* T;
  long long nb, rows;
  __device__ double operator()(long long r, long long k) const {
    if (r >= rows || k >= nb) return 0.0;
    const long long P = r / nb, pp = r - P * nb;
    return T[(P * nb + k) * nb + pp];
  }
};

}  // namespace

size_t fx_ab_bytes(int nb, int na, long long nov) {
  const long long nbp = fx_pad(nb), nap = fx_pad(na);
  return fx_mat_bytes(nb, nbp) + fx_mat_bytes((long long)na * nb, nbp) + fx_mat_bytes(nov, nap) + 1024;
}

// (a) on the fixed-point engine: T[P][mu][q] = sum_nu L[P][mu][nu] C[nu][q], then
// B[P][p][q] = sum_mu T[P][mu][p] C[mu][q] (= (C^T L_P C)[q][p], B_P symmetric).
int stage_ri_mo_transform_fx(Exec& ex, MolBuf& m, const FxMat& L, void* arena) {
  const int nb = m.nb, na = m.na;
  const long long nbp = fx_pad(nb), rows = (long long)na * nb;
  char* p = (char*)arena;
  FxMat Cb = fx_mat_carve(p, nb, nbp);                     // (q, nu) = C[nu][q]
  p += fx_mat_bytes(nb, nbp);
  FxMat Ta = fx_mat_carve(p, rows, nbp);                   // ((P, p), mu) = T[P][mu][p]
  fx_split(ex, m.C, nb, nb, 1, nb, nullptr, Cb);
  FxGemm g1;
  g1.M = (int)rows; g1.N = nb; g1.K = (int)nbp;
  g1.A = L; g1.B = Cb;
  g1.out = m.T1; g1.out_ld = nb;
  int r = fx_gemm(ex, g1);
  if (r) return r;
  TSrc ts{m.T1, nb, rows};
  fx_slice(ex, ts, rows, Ta);
  FxGemm g2;
  g2.M = (int)rows; g2.N = nb; g2.K = (int)nbp;
  g2.A = Ta; g2.B = Cb;
  g2.out = m.B; g2.out_ld = nb;
  return fx_gemm(ex, g2);
}

// (b) on the fixed-point engine: M = D^2 + Xv Xv^T, the lower 64-blocks of the
// column-major matrix (diagonal blocks in full), one launch per 1024-wide K group.
int stage_rpa_build_fx(Exec& ex, MolBuf& m, void* arena) {
  const int nb = m.nb, na = m.na;
  const long long nov = m.nov, nbp = fx_pad(nb), nap = fx_pad(na);
  gather_xv(ex, m);                                        // float64 Xv (column-major) and D
  char* p = (char*)arena + fx_mat_bytes(nb, nbp) + fx_mat_bytes((long long)na * nb, nbp);
  FxMat X = fx_mat_carve(p, nov, nap);                     // (t, P) = Xv[P][t]
  fx_split(ex, m.Xv, nov, na, 1, nov, nullptr, X);
  for (long long g0 = 0; g0 < nap; g0 += kFxGroup) {
    FxGemm g;
    g.M = (int)nov; g.N = (int)nov; g.K = (int)std::min<long long>(kFxGroup, nap - g0); g.k0 = (int)g0;
    g.A = X; g.B = X;
    g.out = m.M; g.out_ld = nov; g.col_major = true;
    g.lower_only = true;
    g.accumulate = g0 > 0;
    g.diag = m.D;
    int r = fx_gemm(ex, g);
    if (r) return r;
  }
  return MOLGW_OK;
}

int fx_mblock(int nb, int na, long long nov, bool mp2) {
  const long long sp = fx_pad(nov);
  const long long per_m = (mp2 ? 2 : 1) * (long long)fx_nsplit((int)fx_pad(na)) * nb * nov * 8 +
                          2 * (long long)fx_mat_bytes(nb, sp);
  return (int)std::max<long long>(1, std::min<long long>(nb, kFxBlockBytes / std::max<long long>(per_m, 1)));
}

size_t fx_sigma_bytes(int nb, int na, long long nov, int mb, bool mp2) {
  const long long nap = fx_pad(na), sp = fx_pad(nov);
  size_t t = 0;
  t += fx_mat_bytes((long long)nb * nb, nap);                            // B^T
  t += fx_mat_bytes(nov, nap);                                           // R^T (qsMP2: B_ia^T)
  t += (size_t)fx_nsplit((int)nap) * mb * nb * nov * sizeof(double);     // w of a block
  t += 2 * fx_mat_bytes(nb, (long long)mb * sp) + 1024;                  // sliced w, g*w
  if (mp2) {
    t += (size_t)fx_nsplit((int)nap) * mb * nb * nov * sizeof(double) + 512;   // exchange partners
    t += fx_mat_bytes((long long)nb * nb, nap) + 2048;   // B_occ^T and B_vir^T: nb^2 rows together
  }
  return t;
}

void fx_bufs_carve(FxBufs& f, int nb, int na, long long nov, int mb, void* base, bool mp2, int no) {
  const long long nap = fx_pad(na);
  char* p = (char*)base;
  f.mb = mb;
  f.Bt = fx_mat_carve(p, (long long)nb * nb, nap);
  p += fx_mat_bytes((long long)nb * nb, nap);
  f.Rt = fx_mat_carve(p, nov, nap);
  p += fx_mat_bytes(nov, nap);
  f.wbuf = (double*)p;
  p += (size_t)fx_nsplit((int)nap) * mb * nb * nov * sizeof(double);
  f.wp_base = (void*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
  f.xbuf = nullptr;
  if (mp2) {
    const long long sp = fx_pad(nov);
    const uintptr_t x = (uintptr_t)f.wp_base + 2 * fx_mat_bytes(nb, (long long)mb * sp) + 1024;
    f.xbuf = (double*)((x + 255) & ~(uintptr_t)255);
    const uintptr_t b = (uintptr_t)(f.xbuf + (size_t)fx_nsplit((int)nap) * mb * nb * nov);
    char* q = (char*)((b + 255) & ~(uintptr_t)255);
    f.Bo = fx_mat_carve(q, (long long)nb * no, nap);
    q += fx_mat_bytes((long long)nb * no, nap);
    f.Bv = fx_mat_carve(q, (long long)nb * (nb - no), nap);
  }
}

int stage_sigma_fx(Exec& ex, MolBuf& m, FxBufs& f, Scratch& s, double eta) {
  const int nb = m.nb, na = m.na, no = m.no;
  const long long nov = m.nov, nn = (long long)nb * nb;
  const long long nap = fx_pad(na), sp = fx_pad(nov);
  // R^T: element (s, P) = R[P][s];  B^T: element ((m, p), P) = B[P][m][p]
  fx_split(ex, m.R, nov, na, 1, nov, nullptr, f.Rt);
  fx_split(ex, m.B, nn, na, 1, nn, nullptr, f.Bt);
  const int nsw = fx_nsplit((int)nap);
  const int max_splits = (int)std::max<long long>(1, (long long)s.splitk_cap / std::max<long long>(nn, 1));
  bool first = true;
  for (int m0 = 0; m0 < nb; m0 += f.mb) {
    const int cnt = std::min(f.mb, nb - m0);
    const long long rows = (long long)cnt * nb;
    FxGemm gw;
    gw.M = (int)rows; gw.N = (int)nov; gw.K = (int)nap;
    gw.A = fx_rows(f.Bt, (long long)m0 * nb, rows);
    gw.B = f.Rt;
    gw.out = f.wbuf;
    gw.out_ld = rows;
    gw.split_stride = rows * nov;
    gw.col_major = true;
    int r = fx_gemm(ex, gw);
    if (r) return r;
    // slices of w and g*w over K = (mm, s), rows p
    const long long K = (long long)cnt * sp;
    FxMat W = fx_mat_carve(f.wp_base, nb, K);
    FxMat P = fx_mat_carve((char*)f.wp_base + ((fx_mat_bytes(nb, K) + 255) / 256 * 256), nb, K);
    {
      KScope ks(ex, MOLGW_K_SIGMA);
      const size_t shm = 2 * kSigRows * kFxGroup * sizeof(double);
      cudaFuncSetAttribute(k_fx_sigma_slices, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
      dim3 grid(ceil_div(nb, kSigRows), W.ngroups);
      k_fx_sigma_slices<<<grid, 256, shm, ex.st>>>(f.wbuf, nsw, rows * nov, rows, (int)sp, (int)nov, nb, no, m0, cnt,
                                                   m.eps, m.Om, eta * eta, W, P);
    }
    // S += P W^T over K, at most max_splits K groups per launch
    const long long kmax = (long long)max_splits * kFxGroup;
    for (long long k0 = 0; k0 < K; k0 += kmax) {
      FxGemm gs;
      gs.M = nb; gs.N = nb;
      gs.K = (int)std::min(kmax, K - k0);
      gs.k0 = (int)k0;
      gs.A = P; gs.B = W;
      gs.out = s.splitk;
      gs.out_ld = nb;
      gs.split_stride = nn;
      gs.col_major = true;
      r = fx_gemm(ex, gs);
      if (r) return r;
      fx_reduce_cm(ex, s.splitk, fx_nsplit(gs.K), nn, nb, nb, s.S, nb, first ? 0.0 : 1.0);
      first = false;
    }
  }
  symmetrize(ex, s.S, nb, m.sigc);
  return MOLGW_OK;
}

// element (r = m cq + q, k = P) = B[P][m][q0 + q], q < cq: a column range of every B_P
struct BColSrc {
  const double* B;
  long long nb, q0, cq, rows, na;
  __device__ double operator()(long long r, long long k) const {
    if (r >= rows || k >= na) return 0.0;
    const long long m = r / cq, q = r - m * cq;
    return B[(k * nb + m) * nb + q0 + q];
  }
};

// qsMP2 on the fixed-point engine (BF16X10): per block of summed orbitals m, the
// direct factor (p m|i a) as one GEMM of B^T (rows (m, p)) with B_ia^T, the
// exchange partners of the block's occupied m as one GEMM (rows (i, p) of B^T against
// rows (m, a) of B_vir^T) and of its empty m as another ((a, p) of B^T against (m, i)
// of B_occ^T), so that each operand is read once per block; then k_fx_mp2_slices and
// S += P W^T as in stage_sigma_fx.  Every K sum is exact per 1024-wide group; the
// denominators float64.
int stage_sigma_mp2_fx(Exec& ex, MolBuf& m, FxBufs& f, Scratch& s, double eta) {
  const int nb = m.nb, na = m.na, no = m.no, nv = nb - no;
  const long long nov = m.nov, nn = (long long)nb * nb;
  const long long nap = fx_pad(na), sp = fx_pad(nov);
  if (!f.xbuf) return MOLGW_E_STATE;
  mp2_prepare(ex, m);
  fx_split(ex, m.R, nov, na, 1, nov, nullptr, f.Rt);
  fx_split(ex, m.B, nn, na, 1, nn, nullptr, f.Bt);
  fx_slice(ex, BColSrc{m.B, nb, 0, no, (long long)nb * no, na}, (long long)nb * no, f.Bo, MOLGW_K_SIGMA);
  fx_slice(ex, BColSrc{m.B, nb, no, nv, (long long)nb * nv, na}, (long long)nb * nv, f.Bv, MOLGW_K_SIGMA);
  const int nsw = fx_nsplit((int)nap);
  const int max_splits = (int)std::max<long long>(1, (long long)s.splitk_cap / std::max<long long>(nn, 1));
  bool first = true;
  for (int m0 = 0; m0 < nb; m0 += f.mb) {
    const int cnt = std::min(f.mb, nb - m0);
    const long long rows = (long long)cnt * nb;
    FxGemm gw;
    gw.M = (int)rows; gw.N = (int)nov; gw.K = (int)nap;
    gw.A = fx_rows(f.Bt, (long long)m0 * nb, rows);
    gw.B = f.Rt;
    gw.out = f.wbuf;
    gw.out_ld = rows;
    gw.split_stride = rows * nov;
    gw.col_major = true;
    int r = fx_gemm(ex, gw);
    if (r) return r;
    // X_m at xbuf + mm nb n_ov: [a'][i][p] for occupied m, [i][a'][p] for empty m
    const int cnt_o = std::max(0, std::min(m0 + cnt, no) - m0);
    const int mv0 = std::max(m0, no), cnt_v = m0 + cnt - mv0;
    if (cnt_o > 0) {
      FxGemm gx;
      gx.M = no * nb; gx.N = cnt_o * nv; gx.K = (int)nap;
      gx.A = fx_rows(f.Bt, 0, (long long)no * nb);
      gx.B = fx_rows(f.Bv, (long long)m0 * nv, (long long)cnt_o * nv);
      gx.out = f.xbuf;
      gx.out_ld = (long long)no * nb;
      gx.split_stride = rows * nov;
      gx.col_major = true;
      r = fx_gemm(ex, gx);
      if (r) return r;
    }
    if (cnt_v > 0) {
      FxGemm gx;
      gx.M = nv * nb; gx.N = cnt_v * no; gx.K = (int)nap;
      gx.A = fx_rows(f.Bt, (long long)no * nb, (long long)nv * nb);
      gx.B = fx_rows(f.Bo, (long long)mv0 * no, (long long)cnt_v * no);
      gx.out = f.xbuf + (long long)(mv0 - m0) * nb * nov;
      gx.out_ld = (long long)nv * nb;
      gx.split_stride = rows * nov;
      gx.col_major = true;
      r = fx_gemm(ex, gx);
      if (r) return r;
    }
    const long long K = (long long)cnt * sp;
    FxMat W = fx_mat_carve(f.wp_base, nb, K);
    FxMat P = fx_mat_carve((char*)f.wp_base + ((fx_mat_bytes(nb, K) + 255) / 256 * 256), nb, K);
    {
      KScope ks(ex, MOLGW_K_SIGMA);
      const size_t shm = 2 * kSigRows * kFxGroup * sizeof(double);
      cudaFuncSetAttribute(k_fx_mp2_slices, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
      dim3 grid(ceil_div(nb, kSigRows), W.ngroups);
      k_fx_mp2_slices<<<grid, 256, shm, ex.st>>>(f.wbuf, f.xbuf, nsw, rows * nov, rows, (int)sp, (int)nov, nb, no,
                                                 m0, cnt, m.eps, m.Om, eta * eta, W, P);
    }
    const long long kmax = (long long)max_splits * kFxGroup;
    for (long long k0 = 0; k0 < K; k0 += kmax) {
      FxGemm gs;
      gs.M = nb; gs.N = nb;
      gs.K = (int)std::min(kmax, K - k0);
      gs.k0 = (int)k0;
      gs.A = P; gs.B = W;
      gs.out = s.splitk;
      gs.out_ld = nb;
      gs.split_stride = nn;
      gs.col_major = true;
      r = fx_gemm(ex, gs);
      if (r) return r;
      fx_reduce_cm(ex, s.splitk, fx_nsplit(gs.K), nn, nb, nb, s.S, nb, first ? 0.0 : 1.0);
      first = false;
    }
  }
  symmetrize(ex, s.S, nb, m.sigc);
  return MOLGW_OK;
}

}  // namespace molgw
