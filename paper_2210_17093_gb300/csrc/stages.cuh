// Per-molecule device buffers and the stage drivers of one RI-qsGW pass.
#pragma once
#include <memory>

#include "common.cuh"
#include "fx.cuh"
#include "tc.cuh"

namespace molgw {

struct MolBuf {
  int nb = 0, na = 0, no = 0;
  int alloc_no = 0;            // n_occ the orbital-size buffers were allocated for
  long long nov = 0;
  bool have_ri = false, have_orb = false;
  bool h_ready = false;        // hmo holds h in the basis of the current MOs
  bool b_valid = false;        // B for the current orbitals
  bool jx_valid = false;       // J, Sigma_x for the current orbitals
  bool rpa_valid = false;      // Omega, R (and ZT) for the current orbitals
  bool sigma_valid = false;    // Sigma_c for the current orbitals
  bool have_b = false, have_rpa = false, have_jx = false, have_sigma = false;  // ever computed
  // inputs / state
  double *L = nullptr, *eps = nullptr, *C = nullptr, *hmo = nullptr;
  // intermediates
  double *B = nullptr, *T1 = nullptr;          // n_aux x nb x nb each
  double *Xv = nullptr, *D = nullptr;          // n_ov x n_aux (column-major), n_ov
  double *M = nullptr, *ZT = nullptr;          // n_ov x n_ov each
  double *Om = nullptr, *R = nullptr;          // n_ov, n_aux x n_ov
  double *XpY = nullptr;                       // n_ov x n_ov (FULL_XPY only)
  double *J = nullptr, *sigx = nullptr, *sigc = nullptr;  // nb x nb
  double* g0w0 = nullptr;                      // G0W0: [eps_QP | Z | Sigma_c,pp(eps_p)], 3 nb
  bool have_g0w0 = false;
  std::vector<void*> ri_allocs, orb_allocs;
  // Open shell (molgw_b200_set_orbitals_open): this MolBuf is the spin-up channel and
  // holds the RPA of both spins (nov = nov_up + n_ov of spin down transitions, up
  // first); dn is the spin-down channel, whose R, Om and D point into this one.
  std::unique_ptr<MolBuf> dn;
  long long nov_up = 0;
};

// Split operands of the tensor-core path (hi/lo pairs, K-major, padded).  L is
// kept per molecule (it changes only with set_ri); the orbital-size operands are
// rebuilt in every pass and are carved from the arena of the lane running it.
struct TcBufs {
  int prec = TC_BF16X3;
  int mb = 0;            // m values per self-energy block
  long long sp = 0;      // padded n_ov
  TcMat L;               // (n_aux*nb) x nb: L[P][nu][mu]       (per set_ri)
  FxMat Lfx;             // the same as 4 fixed-point digits (BF16X10 with MOLGW_FLAG_TC_AB)
  TcMat Ct, X, Xv, Rt, Bt, W, P;                  // per pass (lane arena)
  float* wpart = nullptr;                         // float32 K-chunk partials of w
  long long wpart_floats = 0;
  std::vector<void*> ri_allocs;
};

size_t tc_ri_doubles(int prec, int nb, int na);
size_t tc_orb_doubles(int prec, int nb, int na, long long nov, int mb);
void tc_ri_carve(TcBufs& t, int prec, int nb, int na, double* base);
void tc_bufs_carve(TcBufs& t, int prec, int nb, int na, long long nov, int mb, double* base);

// Operands of the fixed-point path (d)+(e): B^T and R^T sliced once per pass,
// w (float64, per block of m) and the sliced w and g*w of the block.
struct FxBufs {
  int mb = 0;                  // m values per block
  FxMat Bt, Rt;                // rows (m, p) and s, K = P
  double* wbuf = nullptr;      // w of a block: [K group][s][(m, p)]
  void* wp_base = nullptr;     // arena of the sliced w and g*w of a block
  double* xbuf = nullptr;      // qsMP2: the exchange partners of a block, per K group
  FxMat Bo, Bv;                // qsMP2: rows (m, i) and (m, a) of B^T, K = P
};
// m values per block; mp2 adds the exchange partners' float64 partials to each block
int fx_mblock(int nb, int na, long long nov, bool mp2 = false);
// lane arena of stages (a), (b) on the fixed-point engine: C, T = L C and Xv as digits
size_t fx_ab_bytes(int nb, int na, long long nov);
size_t fx_sigma_bytes(int nb, int na, long long nov, int mb, bool mp2 = false);
void fx_bufs_carve(FxBufs& f, int nb, int na, long long nov, int mb, void* base, bool mp2 = false, int no = 0);

struct Scratch {
  double* rho = nullptr;        // n_aux
  double* splitk = nullptr;     // split-K partials
  size_t splitk_cap = 0;        // doubles
  double *wblk = nullptr, *pblk = nullptr;   // w and g-weighted w for a block of m
  size_t wblk_cap = 0;          // doubles per buffer
  double *S = nullptr, *H = nullptr, *U = nullptr;  // nb x nb
  int nb_cap = 0, na_cap = 0;
  void* base = nullptr;
  // packed residues w over the pairs m <= p (float64 path), and the packed B^T
  double *wpk = nullptr, *bpt = nullptr;
  size_t wpk_cap = 0, bpt_cap = 0;
  void* pk_base = nullptr;
};

void dev_copy(Exec& ex, const double* a, double* b, long long n);
void check_finite(Exec& ex, const double* a, long long n);
void fill_upper(Exec& ex, double* M, long long n);
void stage_ri_mo_transform(Exec& ex, MolBuf& m);
// J and Sigma_x of molecule m; with `other` (the other spin channel of an open
// shell) the density of both channels enters J, without the closed-shell factor 2.
void stage_j_sigx(Exec& ex, MolBuf& m, Scratch& s, const MolBuf* other = nullptr);
void stage_rpa_build(Exec& ex, MolBuf& m);
void stage_rpa_eigensolve(Exec& ex, MolBuf& m, EigWork& w, Scratch& s, bool full_xpy);
void stage_sigma(Exec& ex, MolBuf& m, Scratch& s, double eta);
void stage_sigma_mp2(Exec& ex, MolBuf& m, Scratch& s, double eta);
int stage_g0w0(Exec& ex, MolBuf& m, Scratch& s, double eta, int p0, int p1);
void derive_h_from_hf(Exec& ex, MolBuf& m);
void h_ao_to_mo(Exec& ex, MolBuf& m, const double* hao, Scratch& s);
void stage_qs_update(Exec& ex, MolBuf& m, EigWork& w, Scratch& s);
void eigh_dense(Exec& ex, EigWork& w, int n, double* A, double* Z);
void gather_xv(Exec& ex, MolBuf& m);
void symmetrize(Exec& ex, const double* S, int n, double* out);

// tensor-core (split precision) versions of stages (a), (b), (d)+(e)
void tc_split_ri(Exec& ex, MolBuf& m, TcBufs& t);
int stage_ri_mo_transform_tc(Exec& ex, MolBuf& m, TcBufs& t);
int stage_rpa_build_tc(Exec& ex, MolBuf& m, TcBufs& t);
int stage_sigma_tc(Exec& ex, MolBuf& m, TcBufs& t, Scratch& s, double eta);
int stage_sigma_fx(Exec& ex, MolBuf& m, FxBufs& f, Scratch& s, double eta);
int stage_sigma_mp2_fx(Exec& ex, MolBuf& m, FxBufs& f, Scratch& s, double eta);
void mp2_prepare(Exec& ex, MolBuf& m);
int stage_ri_mo_transform_fx(Exec& ex, MolBuf& m, const FxMat& L, void* arena);
int stage_rpa_build_fx(Exec& ex, MolBuf& m, void* arena);

}  // namespace molgw
