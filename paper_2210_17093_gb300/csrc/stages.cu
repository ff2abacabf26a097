// Stage kernels of one RI-qsGW pass (float64 path) and their drivers.
#include <math.h>

#include "stages.cuh"

namespace molgw {

namespace {

__device__ __forceinline__ long long gtid() { return blockIdx.x * (long long)blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

inline int grid_for(long long n, int bs = 256) {
  return (int)std::max<long long>(1, std::min<long long>((n + bs - 1) / bs, 152LL * 32));
}

// Xv[t + P*n_ov] = 2 sqrt(D_t) B[P][i][a]  (t = i*nv + a - no), D[t] = eps_a - eps_i.
__global__ void k_gather_xv(const double* B, const double* eps, int nb, int no, int na,
                            double* Xv, double* D) {
  const int nv = nb - no;
  const long long nov = (long long)no * nv;
  const long long total = nov * na;
  for (long long idx = gtid(); idx < total; idx += gstride()) {
    const long long t = idx % nov;
    const int P = (int)(idx / nov);
    const int i = (int)(t / nv), a = no + (int)(t % nv);
    const double Dt = eps[a] - eps[i];
    if (P == 0) D[t] = Dt;
    Xv[idx] = 2.0 * sqrt(Dt) * B[(long long)P * nb * nb + (long long)i * nb + a];
  }
}

// Open shell: rows t0 .. t0 + no*nv - 1 of Xv = sqrt(2) D^1/2 B_ia^T (n_tot x n_aux,
// column-major) and of D for one spin channel (the spin sum of the closed-shell
// factor 2 is written out over the two channels).
__global__ void k_gather_xv_spin(const double* B, const double* eps, int nb, int no, int na, long long t0,
                                 long long ntot, double* Xv, double* D) {
  const int nv = nb - no;
  const long long nov = (long long)no * nv;
  const long long total = nov * na;
  for (long long idx = gtid(); idx < total; idx += gstride()) {
    const long long t = idx % nov;
    const int P = (int)(idx / nov);
    const int i = (int)(t / nv), a = no + (int)(t % nv);
    const double Dt = eps[a] - eps[i];
    if (P == 0) D[t0 + t] = Dt;
    Xv[t0 + t + (long long)P * ntot] = sqrt(2.0 * Dt) * B[(long long)P * nb * nb + (long long)i * nb + a];
  }
}

__global__ void k_add_diag_sq(double* M, const double* D, long long n) {
  for (long long t = gtid(); t < n; t += gstride()) M[t + t * n] += D[t] * D[t];
}

// Omega = sqrt(lambda); status NUMERIC if lambda <= 0 or not finite.
__global__ void k_omega(const double* lam, double* Om, int n, int* status) {
  for (long long s = gtid(); s < n; s += gstride()) {
    const double l = lam[s];
    if (!(l > 0.0) || !isfinite(l)) { set_status(status, MOLGW_E_NUMERIC); Om[s] = 0.0; }
    else Om[s] = sqrt(l);
  }
}

// R[P][s] *= 1 / sqrt(2 Omega_s)
__global__ void k_scale_r(double* R, const double* Om, int na, int nov) {
  const long long total = (long long)na * nov;
  for (long long idx = gtid(); idx < total; idx += gstride()) {
    const int s = (int)(idx % nov);
    const double o = Om[s];
    R[idx] = (o > 0.0) ? R[idx] / sqrt(2.0 * o) : 0.0;
  }
}

// (X+Y)[t][s] = sqrt(2 D_t / Omega_s) Z[t][s] with the gauge of column s fixed
// (largest |Z[t][s]| positive).  Z row-major n x n; one thread per column.
__global__ void k_xpy(const double* Z, const double* D, const double* Om, int n, double* X) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  double big = -1.0, sg = 1.0;
  for (int t = 0; t < n; ++t) {
    const double z = Z[(long long)t * n + s];
    if (fabs(z) > big) { big = fabs(z); sg = (z >= 0.0) ? 1.0 : -1.0; }
  }
  const double o = Om[s];
  for (int t = 0; t < n; ++t)
    X[(long long)t * n + s] = sg * sqrt(2.0 * D[t] / o) * Z[(long long)t * n + s];
}

// Bo[p][P*no + i] = B[P][p][i]
__global__ void k_gather_bocc(const double* B, int nb, int no, int na, double* Bo) {
  const long long K = (long long)na * no;
  const long long total = (long long)nb * K;
  for (long long idx = gtid(); idx < total; idx += gstride()) {
    const int p = (int)(idx / K);
    const long long k = idx % K;
    const int P = (int)(k / no), i = (int)(k % no);
    Bo[idx] = B[(long long)P * nb * nb + (long long)p * nb + i];
  }
}

// rho_P = sum_i B[P][i][i]
__global__ void k_rho(const double* B, int nb, int no, int na, double* rho) {
  for (long long P = gtid(); P < na; P += gstride()) {
    double s = 0.0;
    for (int i = 0; i < no; ++i) s += B[P * nb * nb + (long long)i * nb + i];
    rho[P] = s;
  }
}

// rho_P += sum_{i < no} B[P][i][i] (the other spin channel of an open shell)
__global__ void k_rho_add(const double* B, int nb, int no, int na, double* rho) {
  for (long long P = gtid(); P < na; P += gstride()) {
    double s = 0.0;
    for (int i = 0; i < no; ++i) s += B[P * nb * nb + (long long)i * nb + i];
    rho[P] += s;
  }
}

// J[pq] = f sum_P B[P][pq] rho_P (f = 2 for a closed shell, 1 with both spins in rho)
__global__ void k_hartree(const double* B, const double* rho, int nb, int na, double f, double* J) {
  const long long nn = (long long)nb * nb;
  for (long long pq = gtid(); pq < nn; pq += gstride()) {
    double s = 0.0;
    for (int P = 0; P < na; ++P) s += B[(long long)P * nn + pq] * rho[P];
    J[pq] = f * s;
  }
}

// Pb[p][mm][s] = Wb[p][mm][s] * g(eps_p - eps_m -/+ Omega_s), m = m0 + mm.
// The shift is +Omega_s for an occupied m (pole eps_i - Omega_s), -Omega_s for a
// virtual m; the subtraction is float64 and g(x) = x / (x^2 + eta^2).
__global__ void k_apply_g(const double* Wb, const double* eps, const double* Om, int nb, int no,
                          int m0, int mb, int nov, double eta, double* Pb) {
  const long long K = (long long)mb * nov;
  const long long total = (long long)nb * K;
  const double eta2 = eta * eta;
  for (long long idx = gtid(); idx < total; idx += gstride()) {
    const int p = (int)(idx / K);
    const long long k = idx % K;
    const int mm = (int)(k / nov), s = (int)(k % nov);
    const int m = m0 + mm;
    const double x = (m < no) ? (eps[p] - eps[m]) + Om[s] : (eps[p] - eps[m]) - Om[s];
    Pb[idx] = Wb[idx] * (x / (x * x + eta2));
  }
}

// Packed pairs m <= p, row-major over m: k(m, p) = m*nb - m(m-1)/2 + (p - m).
__device__ __forceinline__ long long pair_index(int m, int p, int nb) {
  if (m > p) { const int t = m; m = p; p = t; }
  return (long long)m * nb - (long long)m * (m - 1) / 2 + (p - m);
}

// BpT[P][k] = B[P][m][p] for the packed pairs k = (m <= p).
__global__ void k_gather_bpair(const double* B, int nb, int na, double* BpT) {
  const long long npair = (long long)nb * (nb + 1) / 2;
  const long long nn = (long long)nb * nb;
  const long long total = npair * na;
  for (long long idx = gtid(); idx < total; idx += gstride()) {
    const long long k = idx % npair;
    const int P = (int)(idx / npair);
    // row m of the packed triangle holding k
    int m = (int)((2.0 * nb + 1.0 - sqrt((2.0 * nb + 1.0) * (2.0 * nb + 1.0) - 8.0 * (double)k)) * 0.5);
    if (m < 0) m = 0;
    while (m > 0 && (long long)m * nb - (long long)m * (m - 1) / 2 > k) --m;
    while ((long long)(m + 1) * nb - (long long)(m + 1) * m / 2 <= k) ++m;
    const int p = m + (int)(k - ((long long)m * nb - (long long)m * (m - 1) / 2));
    BpT[idx] = B[(long long)P * nn + (long long)m * nb + p];
  }
}

// Wb[p][mm][s] = w^s_{p m} from the packed residues (w symmetric in p, m), and
// Pb = Wb * g(eps_p - eps_m -/+ Omega_s) (float64 subtraction), m = m0 + mm.
__global__ void k_gather_w_apply_g(const double* Wpk, const double* eps, const double* Om, int nb, int no, int m0,
                                   int mb, int nov, double eta, double* Wb, double* Pb) {
  const long long K = (long long)mb * nov;
  const long long total = (long long)nb * K;
  const double eta2 = eta * eta;
  for (long long idx = gtid(); idx < total; idx += gstride()) {
    const int p = (int)(idx / K);
    const long long k = idx % K;
    const int mm = (int)(k / nov), sidx = (int)(k % nov);
    const int m = m0 + mm;
    const double w = Wpk[pair_index(m, p, nb) * nov + sidx];
    const double x = (m < no) ? (eps[p] - eps[m]) + Om[sidx] : (eps[p] - eps[m]) - Om[sidx];
    Wb[idx] = w;
    Pb[idx] = w * (x / (x * x + eta2));
  }
}

// qsMP2: Bia[P][t] = B^P_ia and D_t = eps_a - eps_i for t = i*nv + (a - no).
__global__ void k_mp2_bia(const double* B, const double* eps, int nb, int no, int na, double* Bia,
                          double* D) {
  const int nv = nb - no;
  const long long nov = (long long)no * nv;
  const long long nn = (long long)nb * nb;
  const long long total = nov * na;
  for (long long idx = gtid(); idx < total; idx += gstride()) {
    const int P = (int)(idx / nov);
    const long long t = idx % nov;
    const int i = (int)(t / nv), a = no + (int)(t % nv);
    Bia[idx] = B[P * nn + (long long)i * nb + a];
    if (P == 0) D[t] = eps[a] - eps[i];
  }
}

// qsMP2, Eq. (Sigma.c.MP2) with the frequency on row p: Pb (holding the exchange
// partner X_m[p][t] on entry) <- g(eps_p - eps_m +/- D_t) (2 A_m[p][t] - X_m[p][t]),
// A_m[p][t] = (p m|i a) in Wb; + D_t for occupied m (2h1p), - D_t for empty m (2p1h).
__global__ void k_apply_g_mp2(const double* Wb, const double* eps, const double* D, int nb, int no, int m0,
                              int mb, int nov, double eta, double* Pb) {
  const long long K = (long long)mb * nov;
  const long long total = (long long)nb * K;
  const double eta2 = eta * eta;
  for (long long idx = gtid(); idx < total; idx += gstride()) {
    const int p = (int)(idx / K);
    const long long k = idx % K;
    const int mm = (int)(k / nov), t = (int)(k % nov);
    const int m = m0 + mm;
    const double x = (m < no) ? (eps[p] - eps[m]) + D[t] : (eps[p] - eps[m]) - D[t];
    Pb[idx] = (2.0 * Wb[idx] - Pb[idx]) * (x / (x * x + eta2));
  }
}

// G0W0, the diagonal of Eq. (Sigma.c.GW): for row p of one block of m (one CTA per
// p), sum over (m, s) of (w^s_pm)^2 g(x) and (w^s_pm)^2 g'(x), x = eps_p - eps_m +/- Omega_s,
// g' = (eta^2 - x^2) / (x^2 + eta^2)^2.  Fixed-order block reduction.
__global__ void k_g0w0_block(const double* Wb, const double* eps, const double* Om, int nb, int no, int p0,
                             int m0, int mb, int nov, double eta, double* part) {
  const int pl = blockIdx.x, p = p0 + pl, np = gridDim.x;
  const long long K = (long long)mb * nov;
  const double eta2 = eta * eta;
  const double* w = Wb + (long long)pl * K;
  double a = 0.0, d = 0.0;
  for (long long k = threadIdx.x; k < K; k += blockDim.x) {
    const int mm = (int)(k / nov), s = (int)(k % nov);
    const int m = m0 + mm;
    const double x = (m < no) ? (eps[p] - eps[m]) + Om[s] : (eps[p] - eps[m]) - Om[s];
    const double q = x * x + eta2;
    const double w2 = w[k] * w[k];
    a += w2 * (x / q);
    d += w2 * ((eta2 - x * x) / (q * q));
  }
  __shared__ double sa[256], sd[256];
  sa[threadIdx.x] = a;
  sd[threadIdx.x] = d;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      sa[threadIdx.x] += sa[threadIdx.x + h];
      sd[threadIdx.x] += sd[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[pl] = sa[0];
    part[np + pl] = sd[0];
  }
}

// Linearised quasiparticle equation: Z_p = 1 / (1 - Sigma'_pp), v_pp = eps_p - h_pp - J_pp,
// eps^QP_p = eps_p + Z_p (Sigma_x,pp + Sigma_c,pp - v_pp), for p0 <= p < p0 + np.
// out = [eps^QP | Z | Sigma_c,pp], each of length nb, indexed by p.
__global__ void k_g0w0_final(const double* part, int nblk, const double* eps, const double* hmo,
                             const double* J, const double* sigx, int nb, int p0, int np, double* out) {
  const int pl = blockIdx.x * blockDim.x + threadIdx.x;
  if (pl >= np) return;
  const int p = p0 + pl;
  double sg = 0.0, dg = 0.0;
  for (int b = 0; b < nblk; ++b) {
    sg += part[2LL * b * np + pl];
    dg += part[2LL * b * np + np + pl];
  }
  const long long pp = (long long)p * nb + p;
  const double v = eps[p] - hmo[pp] - J[pp];
  const double z = 1.0 / (1.0 - dg);
  out[p] = eps[p] + z * (sigx[pp] + sg - v);
  out[nb + p] = z;
  out[2 * nb + p] = sg;
}

// out = 1/2 (S + S^T)
__global__ void k_symmetrize(const double* S, int n, double* out) {
  const long long nn = (long long)n * n;
  for (long long idx = gtid(); idx < nn; idx += gstride()) {
    const int p = (int)(idx / n), q = (int)(idx % n);
    out[idx] = 0.5 * (S[idx] + S[(long long)q * n + p]);
  }
}

// h = diag(eps) - J - Sx
__global__ void k_hf_core(const double* eps, const double* J, const double* Sx, int n, double* h) {
  const long long nn = (long long)n * n;
  for (long long idx = gtid(); idx < nn; idx += gstride()) {
    const int p = (int)(idx / n), q = (int)(idx % n);
    h[idx] = ((p == q) ? eps[p] : 0.0) - J[idx] - Sx[idx];
  }
}

// H = 1/2 [(h + J + Sx + Sc) + (.)^T], written column-major (= row-major, symmetric).
__global__ void k_build_h(const double* h, const double* J, const double* Sx, const double* Sc, int n,
                          double* H) {
  const long long nn = (long long)n * n;
  for (long long idx = gtid(); idx < nn; idx += gstride()) {
    const int p = (int)(idx / n), q = (int)(idx % n);
    const long long tr = (long long)q * n + p;
    const double a = h[idx] + J[idx] + Sx[idx] + Sc[idx];
    const double b = h[tr] + J[tr] + Sx[tr] + Sc[tr];
    H[idx] = 0.5 * (a + b);
  }
}

// Fix the sign of each column of U (row-major n x n): largest |entry| positive.
__global__ void k_gauge_cols(double* U, int n) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  double big = -1.0, sg = 1.0;
  for (int t = 0; t < n; ++t) {
    const double z = U[(long long)t * n + s];
    if (fabs(z) > big) { big = fabs(z); sg = (z >= 0.0) ? 1.0 : -1.0; }
  }
  if (sg < 0.0)
    for (int t = 0; t < n; ++t) U[(long long)t * n + s] = -U[(long long)t * n + s];
}

__global__ void k_copy(const double* a, double* b, long long n) {
  for (long long i = gtid(); i < n; i += gstride()) b[i] = a[i];
}

// M[t + u*n] = M[u + t*n] for u > t (copy the lower triangle to the upper one).
__global__ void k_fill_upper(double* M, long long n) {
  const long long total = n * n;
  for (long long idx = gtid(); idx < total; idx += gstride()) {
    const long long t = idx % n, u = idx / n;
    if (u > t) M[idx] = M[u + t * n];
  }
}

__global__ void k_check_finite(const double* a, long long n, int* status) {
  for (long long i = gtid(); i < n; i += gstride())
    if (!isfinite(a[i])) { set_status(status, MOLGW_E_NUMERIC); return; }
}

}  // namespace

void dev_copy(Exec& ex, const double* a, double* b, long long n) {
  KScope ks(ex, MOLGW_K_MISC);
  k_copy<<<grid_for(n), 256, 0, ex.st>>>(a, b, n);
}

void fill_upper(Exec& ex, double* M, long long n) {
  KScope ks(ex, MOLGW_K_MISC);
  k_fill_upper<<<grid_for(n * n), 256, 0, ex.st>>>(M, n);
}

void check_finite(Exec& ex, const double* a, long long n) {
  KScope ks(ex, MOLGW_K_MISC);
  k_check_finite<<<grid_for(n), 256, 0, ex.st>>>(a, n, ex.status);
}

// (a) B[P] = C^T L[P] C as two float64 GEMMs (through T1[P][mu][q]).
void stage_ri_mo_transform(Exec& ex, MolBuf& m) {
  const int nb = m.nb, na = m.na;
  const long long nn = (long long)nb * nb;
  GemmF64 g1;
  g1.M = na * nb; g1.N = nb; g1.K = nb;
  g1.A = m.L; g1.sa_m = nb; g1.sa_k = 1;
  g1.B = m.C; g1.sb_k = nb; g1.sb_n = 1;
  g1.C = m.T1; g1.sc_m = nb; g1.sc_n = 1;
  gemm_f64(ex, g1);
  GemmF64 g2;
  g2.M = nb; g2.N = nb; g2.K = nb; g2.batch = na;
  g2.A = m.C; g2.sa_m = 1; g2.sa_k = nb; g2.sa_b = 0;          // C^T
  g2.B = m.T1; g2.sb_k = nb; g2.sb_n = 1; g2.sb_b = nn;
  g2.C = m.B; g2.sc_m = nb; g2.sc_n = 1; g2.sc_b = nn;
  gemm_f64(ex, g2);
}

// Hartree J and exchange Sigma_x from B (Eqs. J, K in the MO basis).
void stage_j_sigx(Exec& ex, MolBuf& m, Scratch& s, const MolBuf* other) {
  const int nb = m.nb, na = m.na, no = m.no;
  {
    KScope ks(ex, MOLGW_K_MISC, other ? 4 : 3);
    k_rho<<<grid_for(na), 256, 0, ex.st>>>(m.B, nb, no, na, s.rho);
    if (other) k_rho_add<<<grid_for(na), 256, 0, ex.st>>>(other->B, nb, other->no, na, s.rho);
    k_hartree<<<grid_for((long long)nb * nb), 256, 0, ex.st>>>(m.B, s.rho, nb, na, other ? 1.0 : 2.0, m.J);
    if (no > 0) k_gather_bocc<<<grid_for((long long)nb * na * no), 256, 0, ex.st>>>(m.B, nb, no, na, m.T1);
  }
  if (no == 0) {   // an empty spin channel has no exchange
    cudaMemsetAsync(m.sigx, 0, sizeof(double) * nb * nb, ex.st);
    return;
  }
  const long long K = (long long)na * no;
  GemmF64 g;
  g.M = nb; g.N = nb; g.K = (int)K;
  g.A = m.T1; g.sa_m = K; g.sa_k = 1;
  g.B = m.T1; g.sb_k = 1; g.sb_n = K;
  g.C = m.sigx; g.sc_m = nb; g.sc_n = 1;
  g.alpha = -1.0;
  g.ksplit = gemm_f64_pick_split(nb, nb, (int)K, 1, s.splitk_cap);
  g.work = s.splitk;
  gemm_f64(ex, g);
}

void gather_xv(Exec& ex, MolBuf& m) {
  if (m.dn) {
    // open shell: spin-up transitions, then spin-down ones
    const MolBuf& d = *m.dn;
    const long long nov_dn = m.nov - m.nov_up;
    KScope ks(ex, MOLGW_K_MISC, 2);
    if (m.nov_up > 0)
      k_gather_xv_spin<<<grid_for(m.nov_up * m.na), 256, 0, ex.st>>>(m.B, m.eps, m.nb, m.no, m.na, 0, m.nov, m.Xv,
                                                                     m.D);
    if (nov_dn > 0)
      k_gather_xv_spin<<<grid_for(nov_dn * m.na), 256, 0, ex.st>>>(d.B, d.eps, m.nb, d.no, m.na, m.nov_up, m.nov,
                                                                   m.Xv, m.D);
    return;
  }
  KScope ks(ex, MOLGW_K_MISC);
  k_gather_xv<<<grid_for(m.nov * m.na), 256, 0, ex.st>>>(m.B, m.eps, m.nb, m.no, m.na, m.Xv, m.D);
}

void symmetrize(Exec& ex, const double* S, int n, double* out) {
  KScope ks(ex, MOLGW_K_MISC);
  k_symmetrize<<<grid_for((long long)n * n), 256, 0, ex.st>>>(S, n, out);
}

// (b) M = diag(D^2) + Xv Xv^T, Xv = 2 D^1/2 B_ia^T (n_ov x n_aux, column-major).
void stage_rpa_build(Exec& ex, MolBuf& m) {
  const int na = m.na;
  const long long nov = m.nov;
  gather_xv(ex, m);
  GemmF64 g;
  g.M = (int)nov; g.N = (int)nov; g.K = na;
  g.A = m.Xv; g.sa_m = 1; g.sa_k = nov;
  g.B = m.Xv; g.sb_k = nov; g.sb_n = 1;
  g.C = m.M; g.sc_m = 1; g.sc_n = nov;
  g.lower_only = true;
  gemm_f64(ex, g);
  KScope ks(ex, MOLGW_K_MISC);
  k_add_diag_sq<<<grid_for(nov), 256, 0, ex.st>>>(m.M, m.D, nov);
}

// (c) eigenpairs of M; Omega; thin back-transformation to R = B^T (X+Y).
void stage_rpa_eigensolve(Exec& ex, MolBuf& m, EigWork& w, Scratch& s, bool full_xpy) {
  const int n = (int)m.nov, na = m.na;
  tridiagonalize(ex, w, n, m.M);
  tridiag_eigvals(ex, w, n);
  {
    KScope ks(ex, MOLGW_K_MISC);
    k_omega<<<grid_for(n), 256, 0, ex.st>>>(w.lam, m.Om, n, ex.status);
  }
  tridiag_eigvecs(ex, w, n, m.ZT, n);
  build_wy(ex, w, n, m.M);
  // Y = Q^T Xv in place (column-major n x na)
  apply_q(ex, w, n, m.M, m.Xv, 1, n, na, 1);
  // R[P][s] = sum_t Y[t][P] ZT[t][s] / sqrt(2 Omega_s)
  if (w.fx && n <= w.fx_rows && na <= w.fx_cols && n >= 128) {
    // on the 7-digit engine: R^T block (s, P) = sum_t ZT(t, s) Y(t, P), written
    // column-major into R; blocks of kFxZBlock eigenvectors, K groups in order
    const long long np = fx_pad(n), nbz = std::min<long long>(n, kFxZBlock);
    char* p = (char*)w.fx;
    p += fx_mat_bytes(64, np, 7);                    // the layout of apply_q's operands:
    FxMat ys = fx_mat_carve(p, na, np, 7);           // Y^T where apply_q kept X^T
    p += fx_mat_bytes(w.fx_cols, np, 7);
    p += fx_mat_bytes(w.fx_rows, 64, 7);
    p += fx_mat_bytes(w.fx_cols, 64, 7);
    fx_split(ex, m.Xv, na, n, n, 1, nullptr, ys, MOLGW_K_BACKTRANSFORM);
    for (long long s0 = 0; s0 < n; s0 += nbz) {
      const int nsb = (int)std::min<long long>(nbz, n - s0);
      FxMat zs = fx_mat_carve(p, nsb, np, 7);
      fx_split(ex, m.ZT + s0, nsb, n, 1, n, nullptr, zs, MOLGW_K_BACKTRANSFORM);
      for (long long g0 = 0; g0 < np; g0 += kFxGroup) {
        FxGemm g;
        g.M = nsb; g.N = na; g.K = (int)std::min<long long>(kFxGroup, np - g0); g.k0 = (int)g0;
        g.A = zs; g.B = ys;
        g.out = m.R + s0; g.out_ld = n; g.col_major = true;
        g.accumulate = g0 > 0;
        g.kclass = MOLGW_K_BACKTRANSFORM;
        fx_gemm(ex, g);
      }
    }
  } else {
    GemmF64 g;
    g.M = na; g.N = n; g.K = n;
    g.A = m.Xv; g.sa_m = n; g.sa_k = 1;
    g.B = m.ZT; g.sb_k = n; g.sb_n = 1;
    g.C = m.R; g.sc_m = n; g.sc_n = 1;
    g.kclass = MOLGW_K_BACKTRANSFORM;
    gemm_f64(ex, g);
  }
  {
    KScope ks(ex, MOLGW_K_MISC);
    k_scale_r<<<grid_for((long long)na * n), 256, 0, ex.st>>>(m.R, m.Om, na, n);
  }
  if (full_xpy && m.XpY) {
    // Z = Q Z_T in place in ZT (row-major), then (X+Y)
    apply_q(ex, w, n, m.M, m.ZT, n, 1, n, 0);
    KScope ks(ex, MOLGW_K_MISC);
    k_xpy<<<ceil_div(n, 128), 128, 0, ex.st>>>(m.ZT, m.D, m.Om, n, m.XpY);
  }
}

// (d)+(e): w per block of m, the g-weighted copy, S += P W^T; Sigma_c = (S + S^T)/2.
void stage_sigma(Exec& ex, MolBuf& m, Scratch& s, double eta) {
  const int nb = m.nb, na = m.na, no = m.no;
  const int nov = (int)m.nov;
  const long long nn = (long long)nb * nb;
  const long long npair = (long long)nb * (nb + 1) / 2;
  const int mb = std::max(1, std::min(nb, (int)(s.wblk_cap / ((long long)nb * nov))));
  const bool packed = s.wpk && s.wpk_cap >= npair * nov && s.bpt_cap >= npair * na;
  if (packed) {
    // w^s_pm = w^s_mp: one GEMM over the pairs m <= p (half of the residue flops)
    {
      KScope ks(ex, MOLGW_K_SIGMA);
      k_gather_bpair<<<grid_for(npair * na), 256, 0, ex.st>>>(m.B, nb, na, s.bpt);
    }
    GemmF64 g;
    g.M = (int)npair; g.N = nov; g.K = na;
    g.A = s.bpt; g.sa_m = 1; g.sa_k = npair;
    g.B = m.R; g.sb_k = nov; g.sb_n = 1;
    g.C = s.wpk; g.sc_m = nov; g.sc_n = 1;
    g.kclass = MOLGW_K_SIGMA;
    gemm_f64(ex, g);
  }
  for (int m0 = 0; m0 < nb; m0 += mb) {
    const int cnt = std::min(mb, nb - m0);
    const long long K = (long long)cnt * nov;
    if (packed) {
      KScope ks(ex, MOLGW_K_SIGMA);
      k_gather_w_apply_g<<<grid_for(nb * K), 256, 0, ex.st>>>(s.wpk, m.eps, m.Om, nb, no, m0, cnt, nov, eta, s.wblk,
                                                               s.pblk);
    } else {
      // Wb[p][mm][s] = sum_P B[P][m][p] R[P][s]
      GemmF64 g;
      g.M = nb; g.N = nov; g.K = na; g.batch = cnt;
      g.A = m.B + (long long)m0 * nb; g.sa_m = 1; g.sa_k = nn; g.sa_b = nb;
      g.B = m.R; g.sb_k = nov; g.sb_n = 1; g.sb_b = 0;
      g.C = s.wblk; g.sc_m = K; g.sc_n = 1; g.sc_b = nov;
      g.kclass = MOLGW_K_SIGMA;
      gemm_f64(ex, g);
      KScope ks(ex, MOLGW_K_SIGMA);
      k_apply_g<<<grid_for(nb * K), 256, 0, ex.st>>>(s.wblk, m.eps, m.Om, nb, no, m0, cnt, nov, eta, s.pblk);
    }
    GemmF64 h;
    h.M = nb; h.N = nb; h.K = (int)K;
    h.A = s.pblk; h.sa_m = K; h.sa_k = 1;
    h.B = s.wblk; h.sb_k = 1; h.sb_n = K;
    h.C = s.S; h.sc_m = nb; h.sc_n = 1;
    h.beta = (m0 == 0) ? 0.0 : 1.0;
    h.ksplit = gemm_f64_pick_split(nb, nb, (int)K, 1, s.splitk_cap);
    h.work = s.splitk;
    h.kclass = MOLGW_K_SIGMA;
    gemm_f64(ex, h);
  }
  KScope ks(ex, MOLGW_K_MISC);
  k_symmetrize<<<grid_for(nn), 256, 0, ex.st>>>(s.S, nb, m.sigc);
}

// qsMP2: B_ia into R ([P][t]) and D_t into Om, the "R" and "Omega" of the residue GEMM.
void mp2_prepare(Exec& ex, MolBuf& m) {
  KScope ks(ex, MOLGW_K_SIGMA);
  k_mp2_bia<<<grid_for((long long)m.na * m.nov), 256, 0, ex.st>>>(m.B, m.eps, m.nb, m.no, m.na, m.R, m.Om);
}

// qsMP2 self-energy, Eqs. (Sigma.c.MP2) and (Sigma.c.qsMP2.real), float64.  Per
// block of summed orbitals m: A_m[p][t] = (p m|i a) (one batched GEMM over the
// block), the exchange partner X_m[p][t] = (m a|i p) for occupied m, (m i|a p) for
// empty m (one GEMM per m, batched over i or a), then
// S += [g (2 A - X)] A^T and Sigma_c = (S + S^T)/2.  Bia and D live in R and Om.
void stage_sigma_mp2(Exec& ex, MolBuf& m, Scratch& s, double eta) {
  const int nb = m.nb, na = m.na, no = m.no, nv = nb - no;
  const int nov = (int)m.nov;
  const long long nn = (long long)nb * nb;
  mp2_prepare(ex, m);
  const int mb = std::max(1, std::min(nb, (int)(s.wblk_cap / ((long long)nb * nov))));
  for (int m0 = 0; m0 < nb; m0 += mb) {
    const int cnt = std::min(mb, nb - m0);
    const long long K = (long long)cnt * nov;
    GemmF64 g;
    g.M = nb; g.N = nov; g.K = na; g.batch = cnt;
    g.A = m.B + (long long)m0 * nb; g.sa_m = 1; g.sa_k = nn; g.sa_b = nb;
    g.B = m.R; g.sb_k = nov; g.sb_n = 1; g.sb_b = 0;
    g.C = s.wblk; g.sc_m = K; g.sc_n = 1; g.sc_b = nov;
    g.kclass = MOLGW_K_SIGMA;
    gemm_f64(ex, g);
    for (int mm = 0; mm < cnt; ++mm) {
      const int mo = m0 + mm;
      GemmF64 e;
      e.M = nb; e.K = na;
      e.sa_m = 1; e.sa_k = nn; e.sa_b = nb;
      e.sb_k = nn; e.sb_n = 1; e.sb_b = 0;
      e.C = s.pblk + (long long)mm * nov; e.sc_m = K;
      e.kclass = MOLGW_K_SIGMA;
      if (mo < no) {
        // X[p][i*nv + a'] = sum_P B^P_ip B^P_{m, no+a'}: batch over i
        e.N = nv; e.batch = no;
        e.A = m.B;
        e.B = m.B + (long long)mo * nb + no;
        e.sc_n = 1; e.sc_b = nv;
      } else {
        // X[p][i*nv + a'] = sum_P B^P_{no+a', p} B^P_{m, i}: batch over a'
        e.N = no; e.batch = nv;
        e.A = m.B + (long long)no * nb;
        e.B = m.B + (long long)mo * nb;
        e.sc_n = nv; e.sc_b = 1;
      }
      gemm_f64(ex, e);
    }
    {
      KScope ks(ex, MOLGW_K_SIGMA);
      k_apply_g_mp2<<<grid_for(nb * K), 256, 0, ex.st>>>(s.wblk, m.eps, m.Om, nb, no, m0, cnt, nov, eta, s.pblk);
    }
    GemmF64 h;
    h.M = nb; h.N = nb; h.K = (int)K;
    h.A = s.pblk; h.sa_m = K; h.sa_k = 1;
    h.B = s.wblk; h.sb_k = 1; h.sb_n = K;
    h.C = s.S; h.sc_m = nb; h.sc_n = 1;
    h.beta = (m0 == 0) ? 0.0 : 1.0;
    h.ksplit = gemm_f64_pick_split(nb, nb, (int)K, 1, s.splitk_cap);
    h.work = s.splitk;
    h.kclass = MOLGW_K_SIGMA;
    gemm_f64(ex, h);
  }
  KScope ks(ex, MOLGW_K_MISC);
  k_symmetrize<<<grid_for(nn), 256, 0, ex.st>>>(s.S, nb, m.sigc);
}

// One-shot G0W0 from the current Omega, R (float64 residues at every precision) for
// the states p0 <= p < p1: w^s_pm for those rows only, per block of m, the diagonal
// sums per block, then the linearised quasiparticle energies into m.g0w0[p].  Needs
// 2 (p1 - p0) ceil(nb / mb) doubles of split-K scratch.
int stage_g0w0(Exec& ex, MolBuf& m, Scratch& s, double eta, int p0, int p1) {
  const int nb = m.nb, na = m.na, no = m.no;
  const int nov = (int)m.nov;
  const long long nn = (long long)nb * nb;
  const int np = p1 - p0;
  if (np <= 0) return MOLGW_OK;
  const int mb = std::max(1, std::min(nb, (int)(s.wblk_cap / ((long long)np * nov))));
  const int nblk = ceil_div(nb, mb);
  if ((size_t)2 * np * nblk > s.splitk_cap) return MOLGW_E_NOMEM;
  for (int b = 0; b < nblk; ++b) {
    const int m0 = b * mb, cnt = std::min(mb, nb - m0);
    const long long K = (long long)cnt * nov;
    // Wb[pl][mm][s] = sum_P B[P][m0 + mm][p0 + pl] R[P][s]: batched over the states of a
    // narrow window (rows m, so that the tiles fill), else over the m of the block
    // (rows p); the same sums in the same order either way
    GemmF64 g;
    g.N = nov; g.K = na;
    g.A = m.B + (long long)m0 * nb + p0; g.sa_k = nn;
    g.B = m.R; g.sb_k = nov; g.sb_n = 1; g.sb_b = 0;
    g.C = s.wblk; g.sc_n = 1;
    if (np < 32) {
      g.M = cnt; g.batch = np;
      g.sa_m = nb; g.sa_b = 1;
      g.sc_m = nov; g.sc_b = K;
    } else {
      g.M = np; g.batch = cnt;
      g.sa_m = 1; g.sa_b = nb;
      g.sc_m = K; g.sc_b = nov;
    }
    g.kclass = MOLGW_K_SIGMA;
    gemm_f64(ex, g);
    KScope ks(ex, MOLGW_K_SIGMA);
    k_g0w0_block<<<np, 256, 0, ex.st>>>(s.wblk, m.eps, m.Om, nb, no, p0, m0, cnt, nov, eta,
                                         s.splitk + 2LL * b * np);
  }
  KScope ks(ex, MOLGW_K_MISC);
  k_g0w0_final<<<ceil_div(np, 128), 128, 0, ex.st>>>(s.splitk, nblk, m.eps, m.hmo, m.J, m.sigx, nb, p0, np,
                                                      m.g0w0);
  return MOLGW_OK;
}

void derive_h_from_hf(Exec& ex, MolBuf& m) {
  KScope ks(ex, MOLGW_K_MISC);
  k_hf_core<<<grid_for((long long)m.nb * m.nb), 256, 0, ex.st>>>(m.eps, m.J, m.sigx, m.nb, m.hmo);
}

// h_MO = C^T h_AO C (h_AO row-major in `hao`, result into m.hmo).
void h_ao_to_mo(Exec& ex, MolBuf& m, const double* hao, Scratch& s) {
  const int nb = m.nb;
  GemmF64 g1;   // tmp = h C
  g1.M = nb; g1.N = nb; g1.K = nb;
  g1.A = hao; g1.sa_m = nb; g1.sa_k = 1;
  g1.B = m.C; g1.sb_k = nb; g1.sb_n = 1;
  g1.C = s.S; g1.sc_m = nb; g1.sc_n = 1;
  gemm_f64(ex, g1);
  GemmF64 g2;   // hmo = C^T tmp
  g2.M = nb; g2.N = nb; g2.K = nb;
  g2.A = m.C; g2.sa_m = 1; g2.sa_k = nb;
  g2.B = s.S; g2.sb_k = nb; g2.sb_n = 1;
  g2.C = m.hmo; g2.sc_m = nb; g2.sc_n = 1;
  gemm_f64(ex, g2);
}

// Dense symmetric eigensolver on the device: A (n x n symmetric, destroyed) ->
// lam (w.lam) and, if Z != NULL, eigenvectors Z row-major (column k = vector k).
void eigh_dense(Exec& ex, EigWork& w, int n, double* A, double* Z) {
  tridiagonalize(ex, w, n, A);
  tridiag_eigvals(ex, w, n);
  if (!Z) return;
  tridiag_eigvecs(ex, w, n, Z, n);
  build_wy(ex, w, n, A);
  apply_q(ex, w, n, A, Z, n, 1, n, 0);
  KScope ks(ex, MOLGW_K_MISC);
  k_gauge_cols<<<ceil_div(n, 128), 128, 0, ex.st>>>(Z, n);
}

// (f) H = h + J + Sx + Sc; H U = U eps'; C' = C U; h' = U^T h U.
void stage_qs_update(Exec& ex, MolBuf& m, EigWork& w, Scratch& s) {
  const int nb = m.nb;
  const long long nn = (long long)nb * nb;
  {
    KScope ks(ex, MOLGW_K_MISC);
    k_build_h<<<grid_for(nn), 256, 0, ex.st>>>(m.hmo, m.J, m.sigx, m.sigc, nb, s.H);
  }
  eigh_dense(ex, w, nb, s.H, s.U);
  dev_copy(ex, w.lam, m.eps, nb);
  GemmF64 g1;   // C' = C U  (into S, then copy)
  g1.M = nb; g1.N = nb; g1.K = nb;
  g1.A = m.C; g1.sa_m = nb; g1.sa_k = 1;
  g1.B = s.U; g1.sb_k = nb; g1.sb_n = 1;
  g1.C = s.S; g1.sc_m = nb; g1.sc_n = 1;
  gemm_f64(ex, g1);
  dev_copy(ex, s.S, m.C, nn);
  GemmF64 g2;   // tmp = h U
  g2.M = nb; g2.N = nb; g2.K = nb;
  g2.A = m.hmo; g2.sa_m = nb; g2.sa_k = 1;
  g2.B = s.U; g2.sb_k = nb; g2.sb_n = 1;
  g2.C = s.S; g2.sc_m = nb; g2.sc_n = 1;
  gemm_f64(ex, g2);
  GemmF64 g3;   // h' = U^T tmp
  g3.M = nb; g3.N = nb; g3.K = nb;
  g3.A = s.U; g3.sa_m = 1; g3.sa_k = nb;
  g3.B = s.S; g3.sb_k = nb; g3.sb_n = 1;
  g3.C = m.hmo; g3.sc_m = nb; g3.sc_n = 1;
  gemm_f64(ex, g3);
}

}  // namespace molgw
