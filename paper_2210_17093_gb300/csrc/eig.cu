// Float64 tridiagonal eigensolver and back-transformation.
//
//  * Eigenvalues: 4 threads per eigenvalue index.  A float32 bisection on the
//    LDL^T pivots q_j = d_j - x - e_{j-1}^2 / q_{j-1} (tiny pivots replaced by
//    -pivmin) brackets it to a few float32 ulps; the float64 phase counts sign
//    changes of the leading principal minors (three-term recurrence with power-
//    of-two rescaling, no division; Barth, Martin and Wilkinson) and takes
//    safeguarded Newton steps on det(T - x I) with the derivative of the same
//    recurrence, each step checked against the Sturm counts of the bracket.
//  * Eigenvectors: for each eigenvalue a twisted factorisation of T - lambda I
//    (Fernando; Parlett and Dhillon): the stationary factor L+ D+ from the top,
//    the progressive factor U- D- from the bottom, the twist index r minimising
//    |gamma_r| = |D+_r + D-_r - (d_r - lambda)|, then z_r = 1 and the two
//    bidiagonal solves outward.  One thread per eigenvector; vector s is stored
//    as the strided column ZT[j*ldz + s] so that a warp reads and writes
//    consecutive addresses at every step.
//  * Back-transformation: compact-WY T factors per 64-column panel (dlarft),
//    then X <- (I - V T^(T) V^T) X panel by panel with float64 GEMMs.
#include <math.h>

#include "common.cuh"
#include "fx.cuh"

namespace molgw {

namespace {

constexpr int NBP = 64;

__global__ void k_gersh(const double* d, const double* e, int n, double* out) {
  // out[0] = lo, out[1] = hi, out[2] = max e^2, out[3] = max |d| + 2 max |e|
  __shared__ double slo[256], shi[256], se[256];
  double lo = INFINITY, hi = -INFINITY, em = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double ea = (k > 0) ? fabs(e[k - 1]) : 0.0;
    const double eb = (k < n - 1) ? fabs(e[k]) : 0.0;
    lo = fmin(lo, d[k] - ea - eb);
    hi = fmax(hi, d[k] + ea + eb);
    if (k < n - 1) em = fmax(em, e[k] * e[k]);
  }
  slo[threadIdx.x] = lo; shi[threadIdx.x] = hi; se[threadIdx.x] = em;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + s]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + s]);
      se[threadIdx.x] = fmax(se[threadIdx.x], se[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nrm = fmax(fabs(slo[0]), fabs(shi[0]));
    const double eps = 2.220446049250313e-16;
    out[0] = slo[0] - 2.0 * eps * nrm * n - 1e-300;
    out[1] = shi[0] + 2.0 * eps * nrm * n + 1e-300;
    out[2] = fmax(se[0], 1e-300) * 2.2250738585072014e-308 * 64.0;  // pivmin
    out[3] = nrm;
  }
}

// Number of eigenvalues of T below x from the three-term recurrence of the leading
// principal minors, p_j = (d_j - x) p_{j-1} - e_{j-1}^2 p_{j-2} (p_{-1} = 1): the
// count of sign changes along p_{-1}, p_0, ..., p_{n-1} (Sturm sequence property),
// with no division.  A zero minor takes the sign opposite to its predecessor (the
// limit of a tiny negative pivot).  The derivatives p_j' follow from the same
// recurrence, and S = p_{n-1}' / p_{n-1} = det'(T - x I) / det(T - x I) gives a
// Newton step x - 1/S.  Every 4 steps the state is rescaled by a power of two, which
// changes neither the signs nor the ratio.  Sign tests and rescaling run on the
// integer pipe; the float64 work is 5 operations per step.
__device__ __forceinline__ int sturm_count_minors(const double* __restrict__ d, const double* __restrict__ e2,
                                                  int n, double x, double* S) {
  double p0 = 1.0, p0d = 0.0;               // p_{j-2}, p_{j-2}'
  double p1 = d[0] - x, p1d = -1.0;         // p_{j-1}, p_{j-1}'
  if (p1 == 0.0) p1 = -1e-300;
  int cnt = (p1 < 0.0);
  for (int j = 1; j < n; ++j) {
    const double dx = d[j] - x;
    const double ee = e2[j - 1];
    double p2 = fma(dx, p1, -ee * p0);
    const double p2d = fma(-ee, p0d, fma(dx, p1d, -p1));
    const long long b1 = __double_as_longlong(p1);
    long long b2 = __double_as_longlong(p2);
    if ((b2 & 0x7fffffffffffffffLL) == 0) {   // zero minor: opposite sign to p_{j-1}
      p2 = (b1 < 0) ? 1e-300 : -1e-300;
      b2 = __double_as_longlong(p2);
    }
    cnt += (int)((unsigned long long)(b1 ^ b2) >> 63);
    p0 = p1; p0d = p1d;
    p1 = p2; p1d = p2d;
    if ((j & 3) == 0) {
      // keep max(|p_{j-2}|, |p_{j-1}|) near 1: multiply the state by 2^-(its exponent)
      const int e1 = (int)((b1 >> 52) & 0x7ff), e2x = (int)((b2 >> 52) & 0x7ff);
      const int ex = (e1 > e2x ? e1 : e2x) - 1023;
      if (ex > 256 || ex < -256) {
        const double f = __longlong_as_double((long long)(1023 - ex) << 52);
        p0 *= f; p0d *= f; p1 *= f; p1d *= f;
      }
    }
  }
  *S = p1d / p1;
  return cnt;
}

__device__ __forceinline__ int sturm_count_f32(const float* __restrict__ d, const float* __restrict__ e2,
                                               int n, float x, float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int cnt = (q < 0.0f);
  for (int j = 1; j < n; ++j) {
    q = d[j] - x - e2[j - 1] / q;
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += (q < 0.0f);
  }
  return cnt;
}

// e2 = e^2 in float64, and float32 copies of d and e^2 for the coarse phase.
__global__ void k_e2(const double* d, const double* e, double* e2, float* d32, float* e232, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n - 1) {
    e2[k] = e[k] * e[k];
    e232[k] = (float)(e[k] * e[k]);
  }
  if (k < n) d32[k] = (float)d[k];
}

// One step of 4-point multisection shared by the 4 lanes of a group: lane l
// evaluates the count at lo + (l+1)(hi-lo)/5; the group keeps the fifth of the
// interval where the count passes k.
template <typename T>
__device__ __forceinline__ void multisect(T& lo, T& hi, int cnt_l, T x_l, int k, int l, unsigned mask) {
  T new_lo = lo, new_hi = hi;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int c = __shfl_sync(mask, cnt_l, m, 4);
    const T x = __shfl_sync(mask, x_l, m, 4);
    if (c <= k) { if (x > new_lo) new_lo = x; }   // eigenvalue k lies above x
    else if (x < new_hi) new_hi = x;              // first point with count > k
  }
  (void)l;
  lo = new_lo;
  hi = new_hi;
}

// Eigenvalue k of T, 4 threads per eigenvalue.  A float32 phase (on the 62x
// faster FP32 pipe) narrows [lo, hi] to a few float32 ulps of ||T||; the bracket
// is widened by a safety margin and accepted only if float64 Sturm counts
// confirm that it still encloses eigenvalue k (else the Gershgorin interval is
// used).  The float64 phase then multisects to 2 eps |lambda| + 4 eps ||T||.
__global__ void __launch_bounds__(32) k_bisect(const double* d, const double* e2, const float* d32,
                                                const float* e232, const double* g, int n, double* lam,
                                                int* status, int max_rounds) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = gt >> 2, l = gt & 3;
  const int lane = threadIdx.x & 31;
  const unsigned mask = 0xFu << (lane & ~3);
  if (k >= n) return;                      // whole groups leave together (n*4 threads are grouped)
  const double glo = g[0], ghi = g[1];
  const double pivmin = g[2], nrm = g[3];
  const double eps = 2.220446049250313e-16;
  const double atol = 4.0 * eps * nrm + 4.0 * pivmin;
  // float32 phase
  const float nrm32 = (float)nrm;
  const float pivmin32 = fmaxf(1e-30f * fmaxf(nrm32 * nrm32, 1.0f), 1e-36f);
  const float tol32 = 16.0f * 5.9604645e-8f * fmaxf(nrm32, 1e-30f);
  float lo32 = (float)glo, hi32 = (float)ghi;
  const bool use32 = nrm > 1e-15 && nrm < 1e15;   // float32 range for d, e^2 and the pivots
  for (int it = 0; use32 && it < 40 && hi32 - lo32 > tol32; ++it) {
    const float x = lo32 + (float)(l + 1) * (hi32 - lo32) * 0.2f;
    const int c = (x > lo32 && x < hi32) ? sturm_count_f32(d32, e232, n, x, pivmin32) : ((x <= lo32) ? 0 : n);
    multisect<float>(lo32, hi32, c, x, k, l, mask);
  }
  const double margin = 64.0 * 5.9604645e-8 * nrm + atol;
  double lo = fmax(glo, (double)lo32 - margin), hi = fmin(ghi, (double)hi32 + margin);
  int cl = 0;
  double S = 0.0;
  if (lo < hi && l < 2) cl = sturm_count_minors(d, e2, n, l == 0 ? lo : hi, &S);
  const int c_lo = __shfl_sync(mask, cl, 0, 4), c_hi = __shfl_sync(mask, cl, 1, 4);
  if (!(lo < hi) || c_lo > k || c_hi <= k) {
    lo = glo;
    hi = ghi;
  }
  // float64 phase: safeguarded Newton on det(T - x I).  While the Newton iterate xn
  // lies inside the bracket, the 4 lanes evaluate xn, xn -/+ e (e = half the last
  // Newton step: the root is there once the iteration converges quadratically) and
  // the bracket midpoint (halving it whatever Newton does); otherwise they
  // multisect.  Every count updates the bracket, which always holds eigenvalue k;
  // the result is the bracket's midpoint once it is 2 eps |lambda| + atol wide.
  bool ok = false;
  double xn = 0.5 * (lo + hi), dn = hi - lo;
  for (int it = 0; it < max_rounds; ++it) {
    const double tol = 2.0 * eps * fmax(fabs(lo), fabs(hi)) + atol;
    if (hi - lo <= tol) { ok = true; break; }
    const bool newton = xn > lo && xn < hi;
    double x;
    if (newton) {
      const double e = fmax(0.5 * fabs(dn), 0.25 * tol);
      x = (l == 0) ? xn : (l == 1) ? xn - e : (l == 2) ? xn + e : 0.5 * (lo + hi);
    } else {
      x = lo + (double)(l + 1) * (hi - lo) * 0.2;
    }
    S = 0.0;
    int c;
    if (x > lo && x < hi)
      c = sturm_count_minors(d, e2, n, x, &S);   // one code path for the whole warp
    else
      c = (x <= lo) ? 0 : n;
    const double plo = lo, phi = hi;
    multisect<double>(lo, hi, c, x, k, l, mask);
    // lane 0's Newton step from its point (ignored when not finite)
    const double S0 = __shfl_sync(mask, S, 0, 4), x0 = __shfl_sync(mask, x, 0, 4);
    const double step = (S0 != 0.0 && isfinite(S0)) ? -1.0 / S0 : 0.0;
    xn = x0 + step;
    dn = step;
    if (!(step != 0.0 && isfinite(xn))) { xn = 0.5 * (lo + hi); dn = hi - lo; }
    if (lo == plo && hi == phi) { ok = true; break; }   // no representable progress
  }
  if (!ok && l == 0) set_status(status, MOLGW_E_NOCONV);
  if (l == 0) lam[k] = 0.5 * (lo + hi);
}

// Twisted factorisation eigenvector of T - lambda_s I; S1/S2 are strided scratch
// columns (element j at [j*ld + s]); the normalised vector is left in S1.
__global__ void __launch_bounds__(32) k_twisted(const double* __restrict__ d, const double* __restrict__ e,
                                                 const double* __restrict__ lam, const double* g, int n,
                                                 double* S1, double* S2, long long ld) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double l = lam[s];
  // guard for zero pivots: a tiny multiple of the matrix scale
  const double piv = fmax(g[3], 1e-300) * 2.220446049250313e-16 * 1e-6 + 1e-300;
  double* z = S1 + s;
  double* u = S2 + s;
  // forward: D+_j into z[j]
  double Dp = d[0] - l;
  if (fabs(Dp) < piv) Dp = piv;
  z[0] = Dp;
  for (int j = 0; j < n - 1; ++j) {
    const double Lp = e[j] / Dp;
    Dp = d[j + 1] - l - Lp * e[j];
    if (fabs(Dp) < piv) Dp = piv;
    z[(long long)(j + 1) * ld] = Dp;
  }
  // backward: U-_j into u[j], gamma_j, twist index.  The stored D+_j are read 8
  // steps ahead of their use (one warp per SM at most: no other latency hiding).
  double Dm = d[n - 1] - l;
  if (fabs(Dm) < piv) Dm = piv;
  double best = fabs(z[(long long)(n - 1) * ld] + Dm - (d[n - 1] - l));
  int r = n - 1;
  constexpr int PF = 8;
  for (int j0 = n - 2; j0 >= 0; j0 -= PF) {
    double zp[PF];
#pragma unroll
    for (int q = 0; q < PF; ++q) zp[q] = (j0 - q >= 0) ? z[(long long)(j0 - q) * ld] : 0.0;
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      const int j = j0 - q;
      if (j < 0) break;
      const double Um = e[j] / Dm;
      u[(long long)j * ld] = Um;
      Dm = d[j] - l - Um * e[j];
      if (fabs(Dm) < piv) Dm = piv;
      const double gam = fabs(zp[q] + Dm - (d[j] - l));
      if (gam < best) { best = gam; r = j; }
    }
  }
  // solve outward from the twist index (stored D+_j and U-_j prefetched likewise)
  double nrm2 = 1.0, big = 1.0;
  int sgn = 1;
  double zj = 1.0;
  for (int j0 = r - 1; j0 >= 0; j0 -= PF) {
    double dp[PF];
#pragma unroll
    for (int q = 0; q < PF; ++q) dp[q] = (j0 - q >= 0) ? z[(long long)(j0 - q) * ld] : 1.0;
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      const int j = j0 - q;
      if (j < 0) break;
      zj = -(e[j] / dp[q]) * zj;
      z[(long long)j * ld] = zj;
      nrm2 += zj * zj;
      if (fabs(zj) > big) { big = fabs(zj); sgn = (zj >= 0.0) ? 1 : -1; }
    }
  }
  z[(long long)r * ld] = 1.0;
  zj = 1.0;
  for (int j0 = r; j0 < n - 1; j0 += PF) {
    double um[PF];
#pragma unroll
    for (int q = 0; q < PF; ++q) um[q] = (j0 + q < n - 1) ? u[(long long)(j0 + q) * ld] : 0.0;
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      const int j = j0 + q;
      if (j >= n - 1) break;
      zj = -um[q] * zj;
      z[(long long)(j + 1) * ld] = zj;
      nrm2 += zj * zj;
      if (fabs(zj) > big) { big = fabs(zj); sgn = (zj >= 0.0) ? 1 : -1; }
    }
  }
  const double sc = (sgn > 0 ? 1.0 : -1.0) / sqrt(nrm2);
  for (int j = 0; j < n; ++j) z[(long long)j * ld] *= sc;
}

// T factor of one panel from its Gram matrix G = V^T V (dlarft, forward, columnwise):
// T(c,c) = tau_c, T(0:c, c) = -tau_c T(0:c, 0:c) G(0:c, c).
__global__ void k_wy_t(const double* Gall, const double* tau, int n, double* Tall) {
  const int p = blockIdx.x;
  const int k0 = p * NBP;
  const int nbp = min(NBP, (n - 1) - k0);
  const double* G = Gall + (long long)p * NBP * NBP;
  double* T = Tall + (long long)p * NBP * NBP;
  __shared__ double Ts[NBP][NBP + 1];
  __shared__ double gcol[NBP];
  const int t = threadIdx.x;  // 64 threads
  for (int r = 0; r < NBP; ++r) Ts[r][t] = 0.0;
  __syncthreads();
  for (int c = 0; c < nbp; ++c) {
    const double tc = tau[k0 + c];
    gcol[t] = (t < c) ? G[t * NBP + c] : 0.0;
    __syncthreads();
    double s = 0.0;
    if (t < c) {
      for (int k = t; k < c; ++k) s += Ts[t][k] * gcol[k];  // T upper triangular
    }
    __syncthreads();
    if (t < c) Ts[t][c] = -tc * s;
    if (t == c) Ts[c][c] = tc;
    __syncthreads();
  }
  for (int r = 0; r < NBP; ++r) T[r * NBP + t] = Ts[r][t];
}

}  // namespace

void eig_work_carve(EigWork& w, double* p, int nmax, int ncols_max) {
  const size_t n = (size_t)std::max(nmax, 2);
  w = EigWork{};
  w.nmax = (int)n;
  w.ncols_max = std::max(ncols_max, 64);
  w.part_cap = eig_part_doubles(n);
  w.gk_cap = eig_gk_doubles(n, (size_t)w.ncols_max);
  const size_t npan = n / 64 + 1;
  w.d = p; p += n; w.e = p; p += n; w.tau = p; p += n; w.lam = p; p += n;
  w.Wp = p; p += n * 64;
  w.part = p; p += w.part_cap;
  w.scal = p; p += 64;
  w.S2 = p; p += n * n;
  w.Tm = p; p += 2 * npan * 64 * 64;   // T factors, then the Gram matrices
  w.tmp1 = p; p += (size_t)64 * w.ncols_max;
  w.tmp2 = p; p += (size_t)64 * w.ncols_max;
  w.gk = p; p += w.gk_cap;
}

int eig_work_alloc(EigWork& w, int nmax, int ncols_max) {
  eig_work_free(w);
  double* p = nullptr;
  const size_t total = eig_work_doubles((size_t)std::max(nmax, 2), (size_t)std::max(ncols_max, 64));
  if (cudaMalloc(&p, total * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return MOLGW_E_NOMEM; }
  eig_work_carve(w, p, nmax, ncols_max);
  w.owned = true;
  return MOLGW_OK;
}

void eig_work_free(EigWork& w) {
  if (w.owned && w.d) cudaFree(w.d);
  w = EigWork{};
}

void tridiag_eigvals(Exec& ex, EigWork& w, int n) {
  double* g = w.scal + 8;       // lo, hi, pivmin, norm
  double* e2 = w.part;          // n-1 squares (the partial-sum area is free after the reduction)
  float* d32 = reinterpret_cast<float*>(w.part + n);
  float* e232 = d32 + n;
  KScope ks(ex, MOLGW_K_BISECT, 3);
  k_gersh<<<1, 256, 0, ex.st>>>(w.d, w.e, n, g);
  k_e2<<<ceil_div(n, 256), 256, 0, ex.st>>>(w.d, w.e, e2, d32, e232, n);
  k_bisect<<<ceil_div(4LL * n, 32), 32, 0, ex.st>>>(w.d, e2, d32, e232, g, n, w.lam, ex.status,
                                                     ex.bisect_rounds);
}

void tridiag_eigvecs(Exec& ex, EigWork& w, int n, double* ZT, long long ldz) {
  KScope ks(ex, MOLGW_K_TWISTED, 1);
  k_twisted<<<ceil_div(n, 32), 32, 0, ex.st>>>(w.d, w.e, w.lam, w.scal + 8, n, ZT, w.S2, ldz);
}

void build_wy(Exec& ex, EigWork& w, int n, const double* A) {
  const int ncols = n - 1;
  if (ncols <= 0) return;
  const int npan = ceil_div(ncols, NBP);
  double* G = w.Tm + (size_t)(w.nmax / NBP + 1) * NBP * NBP;   // npan x 64 x 64 Gram matrices
  // G_p(a, b) = sum_r V_p(r, a) V_p(r, b); V_p = A[:, k0..k0+64) is zero above its
  // unit diagonal, so every full panel is one batch entry of a K = n GEMM.
  const int nfull = (ncols % NBP == 0) ? npan : npan - 1;
  if (nfull > 0) {
    GemmF64 gm;
    gm.M = NBP; gm.N = NBP; gm.K = n; gm.batch = nfull;
    gm.A = A; gm.sa_m = n; gm.sa_k = 1; gm.sa_b = (long long)NBP * n;
    gm.B = A; gm.sb_k = 1; gm.sb_n = n; gm.sb_b = (long long)NBP * n;
    gm.C = G; gm.sc_m = NBP; gm.sc_n = 1; gm.sc_b = NBP * NBP;
    gm.ksplit = gemm_f64_pick_split(NBP, NBP, n, nfull, w.gk_cap);
    gm.work = w.gk;
    gm.kclass = MOLGW_K_BACKTRANSFORM;
    gemm_f64(ex, gm);
  }
  if (nfull < npan) {
    const int k0 = nfull * NBP;
    const int nbp = ncols - k0;
    GemmF64 gm;
    gm.M = nbp; gm.N = nbp; gm.K = n - k0;
    gm.A = A + k0 + (long long)k0 * n; gm.sa_m = n; gm.sa_k = 1;
    gm.B = A + k0 + (long long)k0 * n; gm.sb_k = 1; gm.sb_n = n;
    gm.C = G + (long long)nfull * NBP * NBP; gm.sc_m = NBP; gm.sc_n = 1;
    gm.kclass = MOLGW_K_BACKTRANSFORM;
    gemm_f64(ex, gm);
  }
  KScope ks(ex, MOLGW_K_BACKTRANSFORM, 1);
  k_wy_t<<<npan, NBP, 0, ex.st>>>(G, w.tau, n, w.Tm);
}

namespace {

// Fixed-point layout of the back-transformation operands inside w.fx.
struct BtFx {
  FxMat vt, xs, vr, t2;
};
BtFx bt_fx(const EigWork& w, long long m, int nc) {
  const long long np = fx_pad(w.fx_rows), mp = fx_pad(m);
  char* p = (char*)w.fx;
  BtFx b;
  b.vt = fx_mat_carve(p, 64, mp, 7);
  p += fx_mat_bytes(64, np, 7);
  b.xs = fx_mat_carve(p, nc, mp, 7);
  p += fx_mat_bytes(w.fx_cols, np, 7);
  b.vr = fx_mat_carve(p, m, 64, 7);
  p += fx_mat_bytes(w.fx_rows, 64, 7);
  b.t2 = fx_mat_carve(p, nc, 64, 7);
  return b;
}

// One panel of apply_q on the 7-digit engine: tmp1 = V^T X[k0:, :] (one launch
// per 1024-wide K group, accumulated in order), tmp2 = T^(T) tmp1 in float64,
// X[k0:, :] -= V tmp2.
void apply_panel_fx(Exec& ex, EigWork& w, int n, const double* V, int nbp, int m, double* Xk, long long sr,
                    long long sc, int nc, const double* T, int trans) {
  BtFx b = bt_fx(w, m, nc);
  const int kp = (int)fx_pad(m);
  fx_split(ex, V, nbp, m, n, 1, nullptr, b.vt, MOLGW_K_BACKTRANSFORM);     // (c, r) = V(r, c)
  fx_split(ex, Xk, nc, m, sc, sr, nullptr, b.xs, MOLGW_K_BACKTRANSFORM);   // (col, r) = X(r, col)
  const int ns = fx_nsplit(kp);
  if ((size_t)ns * nbp * nc > w.gk_cap) {
    // partials would not fit: one launch per K group, accumulated in order
    for (int g0 = 0; g0 < kp; g0 += kFxGroup) {
      FxGemm g;
      g.M = nbp; g.N = nc; g.K = std::min(kFxGroup, kp - g0); g.k0 = g0;
      g.A = b.vt; g.B = b.xs;
      g.out = w.tmp1; g.out_ld = nc;
      g.accumulate = g0 > 0;
      g.kclass = MOLGW_K_BACKTRANSFORM;
      fx_gemm(ex, g);
    }
  } else {
    // all K groups in one launch: per-group partials in the split-K workspace,
    // then summed in group order into tmp1
    FxGemm g;
    g.M = nbp; g.N = nc; g.K = kp;
    g.A = b.vt; g.B = b.xs;
    g.out = w.gk; g.out_ld = nc;
    g.split_stride = (long long)nbp * nc;
    g.kclass = MOLGW_K_BACKTRANSFORM;
    fx_gemm(ex, g);
    fx_reduce_rm(ex, w.gk, ns, (long long)nbp * nc, nbp, nc, w.tmp1, nc, 0.0);
  }
  GemmF64 g2;
  g2.M = nbp; g2.N = nc; g2.K = nbp;
  g2.A = T; if (trans) { g2.sa_m = 1; g2.sa_k = NBP; } else { g2.sa_m = NBP; g2.sa_k = 1; }
  g2.B = w.tmp1; g2.sb_k = nc; g2.sb_n = 1;
  g2.C = w.tmp2; g2.sc_m = nc; g2.sc_n = 1;
  g2.kclass = MOLGW_K_BACKTRANSFORM;
  gemm_f64(ex, g2);
  fx_split(ex, V, m, nbp, 1, n, nullptr, b.vr, MOLGW_K_BACKTRANSFORM);      // (r, c) = V(r, c)
  fx_split(ex, w.tmp2, nc, nbp, 1, nc, nullptr, b.t2, MOLGW_K_BACKTRANSFORM);  // (col, c) = tmp2(c, col)
  FxGemm g3;
  g3.M = m; g3.N = nc; g3.K = 64;
  g3.A = b.vr; g3.B = b.t2;
  g3.out = Xk;
  g3.col_major = (sr == 1);
  g3.out_ld = (sr == 1) ? sc : sr;
  g3.accumulate = true;
  g3.alpha = -1.0;
  g3.kclass = MOLGW_K_BACKTRANSFORM;
  fx_gemm(ex, g3);
}

}  // namespace

void apply_q(Exec& ex, EigWork& w, int n, const double* A, double* X, long long sr, long long sc,
             int ncols, int trans) {
  const int nref = n - 1;
  if (nref <= 0 || ncols <= 0) return;
  const int npan = ceil_div(nref, NBP);
  const bool fx = w.fx && n <= w.fx_rows && std::min(ncols, w.ncols_max) <= w.fx_cols && (sr == 1 || sc == 1);
  for (int c0 = 0; c0 < ncols; c0 += w.ncols_max) {
    const int nc = std::min(w.ncols_max, ncols - c0);
    double* Xc = X + (long long)c0 * sc;
    for (int q = 0; q < npan; ++q) {
      const int p = trans ? q : (npan - 1 - q);
      const int k0 = p * NBP;
      const int nbp = std::min(NBP, nref - k0);
      const int m = n - k0;
      const double* V = A + k0 + (long long)k0 * n;     // m x nbp, column-major
      const double* T = w.Tm + (long long)p * NBP * NBP;
      if (fx && m >= 128) {
        apply_panel_fx(ex, w, n, V, nbp, m, Xc + (long long)k0 * sr, sr, sc, nc, T, trans);
        continue;
      }
      // tmp1 (nbp x nc) = V^T X[k0:, :]
      GemmF64 g1;
      g1.M = nbp; g1.N = nc; g1.K = m;
      g1.A = V; g1.sa_m = n; g1.sa_k = 1;
      g1.B = Xc + (long long)k0 * sr; g1.sb_k = sr; g1.sb_n = sc;
      g1.C = w.tmp1; g1.sc_m = nc; g1.sc_n = 1;
      g1.ksplit = gemm_f64_pick_split(nbp, nc, m, 1, w.gk_cap);
      g1.work = w.gk;
      g1.kclass = MOLGW_K_BACKTRANSFORM;
      gemm_f64(ex, g1);
      // tmp2 = T^T tmp1 (Q^T) or T tmp1 (Q)
      GemmF64 g2;
      g2.M = nbp; g2.N = nc; g2.K = nbp;
      g2.A = T; if (trans) { g2.sa_m = 1; g2.sa_k = NBP; } else { g2.sa_m = NBP; g2.sa_k = 1; }
      g2.B = w.tmp1; g2.sb_k = nc; g2.sb_n = 1;
      g2.C = w.tmp2; g2.sc_m = nc; g2.sc_n = 1;
      g2.kclass = MOLGW_K_BACKTRANSFORM;
      gemm_f64(ex, g2);
      // X[k0:, :] -= V tmp2
      GemmF64 g3;
      g3.M = m; g3.N = nc; g3.K = nbp;
      g3.A = V; g3.sa_m = 1; g3.sa_k = n;
      g3.B = w.tmp2; g3.sb_k = nc; g3.sb_n = 1;
      g3.C = Xc + (long long)k0 * sr; g3.sc_m = sr; g3.sc_n = sc;
      g3.alpha = -1.0; g3.beta = 1.0;
      g3.kclass = MOLGW_K_BACKTRANSFORM;
      gemm_f64(ex, g3);
    }
  }
}

}  // namespace molgw
