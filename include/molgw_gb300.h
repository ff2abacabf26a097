/*
 * molgw_gb300.h -- C ABI of the GB300 (sm_103a) RI-qsGW hot path.
 *
 * One closed-shell quasiparticle self-consistent GW iteration (arXiv 2210.17093,
 * Sec. II.C) with the resolution-of-identity factorisation of the Coulomb
 * integrals, split into the stages
 *   (a) ri_mo_transform   B^P_pq = sum_{mu nu} C_{mu p} (P|mu nu) C_{nu q}        Eq. (AO.to.MO)
 *   (b) rpa_build         M = D^2 + 4 D^1/2 K D^1/2, K_tu = sum_P B^P_t B^P_u    Eqs. (Casida.A/B)
 *   (c) rpa_eigensolve    M Z = Z Omega^2, (X+Y) = sqrt(2) D^1/2 Z Omega^-1/2     Eq. (Casida.AB.XY)
 *   (d) gw_residues       w^s_pq = sum_P B^P_pq (B^T (X+Y))_Ps                   Eq. (w.residue)
 *   (e) sigma_assembly    Sigma_x (Eq. K) and the Hermitised Sigma_c
 *                         1/2 Re[Sigma_pq(eps_p) + Sigma_pq(eps_q)]        Eqs. (Sigma.c.GW), (Sigma.c.qsGW.real)
 *   (f) qs_update         H = h + J + Sigma_x + Sigma_c, H U = U eps', C' = C U   Eqs. (H), (GEP), (J)
 *
 * Beside it: qsMP2 (MOLGW_FLAG_QSMP2, Eqs. (Sigma.c.MP2), (Sigma.c.qsMP2.real)),
 * one-shot G0W0 (molgw_b200_g0w0, Sec. II.C) and open shells
 * (molgw_b200_set_orbitals_open, the sigma-resolved equations of Sec. II).
 *
 * Conventions (all entry points)
 *   - Closed shell unless molgw_b200_set_orbitals_open, real orbitals, orthonormal
 *     AO basis (S = I).  Sizes:
 *     nb = n_basis, no = n_occ, nv = nb - no, n_ov = no*nv, na = n_aux.
 *     Transition index t = i*nv + (a - no), occupied-major.
 *   - Every array argument is a plain pointer to float64 data that may live in
 *     host memory (pageable or pinned) or in device memory of the context's
 *     device; the library tells them apart with cudaPointerGetAttributes.
 *     Matrices are row-major: X[r][c] at X[r*ld + c] with ld = the row length.
 *   - Ownership: the caller owns every pointer it passes.  Inputs are copied
 *     into library-owned device memory on the context stream before the call
 *     returns control of the stream; a device input must stay valid until the
 *     stream passes that point.  Outputs are written stream-ordered; for a host
 *     output the call synchronises the stream before it returns.
 *   - Errors: argument and call-order errors are returned at once and change no
 *     state.  Errors found on the device (non-positive RPA eigenvalue, a
 *     non-finite value, an eigensolver iteration cap or a bounded wait that ran
 *     out) are latched in a device status word and returned by the next call
 *     that synchronises (a call with a host output, molgw_b200_sync or
 *     molgw_b200_destroy).
 *   - Batches: mol = -1 runs every ready molecule.  The molecules are spread
 *     over concurrent streams of the context (opts.lanes), which fork from the
 *     context stream and are joined back into it before the call returns, so
 *     that all work stays ordered on the context stream.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef MOLGW_GB300_H
#define MOLGW_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct molgw_ctx_s* molgw_ctx;

enum molgw_status {
  MOLGW_OK = 0,
  MOLGW_E_ARG = -1,      /* bad argument (size, NULL, index out of range)           */
  MOLGW_E_STATE = -2,    /* call out of order (e.g. rpa before set_ri/set_orbitals) */
  MOLGW_E_NOMEM = -3,    /* device allocation failed                                */
  MOLGW_E_CUDA = -4,     /* a CUDA runtime call failed                              */
  MOLGW_E_NOCONV = -5,   /* eigensolver iteration cap reached                       */
  MOLGW_E_TIMEOUT = -6,  /* a bounded device-side wait ran out                      */
  MOLGW_E_NUMERIC = -7   /* non-positive RPA eigenvalue or non-finite value         */
};

/* Arithmetic of the dense contractions (a), (b), (d) and the Sigma_c
 * contraction of (e).  The eigensolvers (c), (f) and the denominators
 * eps_p - eps_m -/+ Omega_s always run in float64. */
enum molgw_precision {
  MOLGW_PREC_FP64 = 0,    /* float64 on the CUDA cores                                   */
  MOLGW_PREC_BF16X3 = 1,  /* tcgen05 BF16 products, 3-term hi/lo split, FP32 accumulate  */
  MOLGW_PREC_TF32X3 = 2,  /* tcgen05 TF32 products, 3-term hi/lo split, FP32 accumulate  */
  MOLGW_PREC_BF16X6 = 3,  /* tcgen05 BF16 products, 3 slices hi+mid+lo, 6 products, FP32 */
  MOLGW_PREC_BF16X10 = 4  /* tcgen05 BF16 products of 4 fixed-point slices (10 products),
                             exact FP32 sums per 256-element chunk, one FP64 rounding per
                             1024-element group; (d) and (e), and (a), (b) with
                             MOLGW_FLAG_TC_AB                                         */
};
/* With BF16X3, TF32X3 or BF16X6 the residue and self-energy contractions (d),
 * (e) run on the tensor cores (the residues in float32 chunks of 64 auxiliary
 * functions summed in float64); (a) and (b) do too only with MOLGW_FLAG_TC_AB.
 * Near a pole (|eps_p - eps_m -/+ Omega_s| ~ eta) Sigma_c responds to an error
 * in Omega_s with a factor up to 1/eta^2, and the split products of (a), (b)
 * leave relative errors of 1e-6 to 1e-5 in M. */

enum molgw_flags {
  MOLGW_FLAG_FULL_XPY = 1u << 0, /* keep the full n_ov x n_ov (X+Y) so molgw_b200_rpa can return it */
  MOLGW_FLAG_KTIMING = 1u << 1,  /* record CUDA events around kernels for molgw_b200_kernel_stats  */
  MOLGW_FLAG_GRAPH = 1u << 2,    /* qs_step from the state a qs_step leaves: captured once into a CUDA
                                    graph (all lanes of mol = -1 in one graph) and replayed while the
                                    buffers and the set of molecules stay the same                  */
  MOLGW_FLAG_USE_STREAM = 1u << 3, /* run on opts.stream even when it is NULL (the legacy default stream) */
  MOLGW_FLAG_TC_AB = 1u << 4,      /* with a split precision: stages (a) and (b) on the tensor cores too */
  MOLGW_FLAG_EIG_TC = 1u << 5,     /* the trailing SYR2K update of the tridiagonalisation and the
                                      back-transformation on the tensor cores: 7 fixed-point BF16
                                      digits per value (56 bits, values within 4x of their group
                                      maximum exact), exact sums, one float64 rounding; and the
                                      panel's mat-vec in fixed point (molgw_b200_set_panel_matvec)
                                      -- float64 accuracy in the normwise sense, not float64
                                      arithmetic; any precision                               */
  MOLGW_FLAG_QSMP2 = 1u << 6       /* qsMP2 instead of qsGW: Sigma_c is the second-order self-energy
                                      of Eq. (Sigma.c.MP2), made static and Hermitian by
                                      Eq. (Sigma.c.qsMP2.real).  Its second-order exchange factor
                                      is (p a|i n) for an occupied summed orbital p (the
                                      antisymmetrised second-order expansion; the printed (p i|a n)
                                      holds for an empty p).  No RPA: sigma and qs_step run (a),
                                      the MP2 residues and (f); rpa, rpa_matrix and the RPA items
                                      return MOLGW_E_STATE.  MOLGW_PREC_FP64, or MOLGW_PREC_BF16X10
                                      (the three contractions on the fixed-point engine, the
                                      denominators float64); other precisions MOLGW_E_ARG at
                                      create                                                   */
};

typedef struct {
  int32_t struct_size; /* sizeof(molgw_opts)                                        */
  int32_t precision;   /* enum molgw_precision                                      */
  int32_t max_mols;    /* molecules the context holds, indices 0 .. max_mols-1 (>=1) */
  int32_t device;      /* CUDA device ordinal                                       */
  double eta;          /* broadening eta > 0 of Eq. (Sigma.c.GW), Hartree           */
  void* stream;        /* cudaStream_t to run on; NULL = a stream the context owns,
                          unless MOLGW_FLAG_USE_STREAM asks for the legacy default stream */
  uint32_t flags;      /* enum molgw_flags                                          */
  int32_t lanes;       /* mol = -1: molecules run on up to this many concurrent streams
                          (at most 16), assigned longest pass first; 0 = 8, or the
                          count molgw_b200_autotune chose                             */
} molgw_opts;

/* Create a context.  Returns MOLGW_E_ARG for a bad opts, MOLGW_E_CUDA if the
 * device cannot be used.  *out is NULL on failure. */
int molgw_b200_create(const molgw_opts* opts, molgw_ctx* out);

/* Three-centre RI factors of molecule `mol`: L[P][mu][nu], n_aux x n_basis x
 * n_basis, symmetric in (mu, nu), already contracted with the Coulomb metric
 * so that (mu nu|la ta) = sum_P L[P][mu][nu] L[P][la][ta] (Sec. II.B names
 * the RI approximation; Eq. (AO.4.ERI) is the integral it factorises).
 * Clears the molecule's orbitals and every result: set_orbitals must follow.
 * n_basis >= 2, n_aux >= 1. */
int molgw_b200_set_ri(molgw_ctx ctx, int mol, int n_basis, int n_aux, const double* L);

/* Orbitals of molecule `mol`: eps[n_basis] ascending MO energies, C[mu][p]
 * (row mu, column = MO p, Eq. (MO)), orthonormal columns.  h_core[mu][nu] is
 * the one-body Hamiltonian T + V_ext of Eq. (H) in the AO basis; NULL reads
 * (eps, C) as a Hartree-Fock solution and derives h_MO = diag(eps) - J - Sigma_x
 * from it at the next pass.  1 <= n_occ < n_basis; set_ri must come first. */
int molgw_b200_set_orbitals(molgw_ctx ctx, int mol, int n_occ, const double* eps,
                            const double* C, const double* h_core);

/* Open shell (float64, or BF16X10 with the fixed-point contractions): the orbitals
 * of molecule `mol` per spin -- n_occ_up, n_occ_dn (0 <= n_occ < n_basis, at least
 * one electron), eps_up/eps_dn[n_basis]
 * ascending, C_up/C_dn[mu][p] orthonormal columns -- for the sigma-resolved
 * equations of Sec. II (Eqs. GEP, H, J, D, K with sigma; Casida.A/B with the spin
 * sum written out: one RPA over the transitions of both spins, spin up first, M =
 * D^2 + 2 D^1/2 K D^1/2, X+Y = D^1/2 Z Omega^-1/2; Eq. w.residue summing sigma'
 * over those transitions; Sigma_c, Sigma_x per spin; J from both spins).  h_core as
 * in set_orbitals (spin independent); NULL reads each spin's (eps, C) as its HF
 * solution.  Afterwards every per-orbital output and fetch item (B, Sigma_x,
 * Sigma_c, J, h_MO, eps, C) is the spin-up block followed by the spin-down block
 * (twice the closed-shell size); Omega and R span the transitions of both spins.
 * MOLGW_E_ARG unless the context is MOLGW_PREC_FP64 or MOLGW_PREC_BF16X10, without
 * MOLGW_FLAG_QSMP2 and MOLGW_FLAG_FULL_XPY; molgw_b200_g0w0 and the G0W0 items
 * return MOLGW_E_STATE for an open-shell molecule.  set_ri or set_orbitals make the molecule closed again. */
int molgw_b200_set_orbitals_open(molgw_ctx ctx, int mol, int n_occ_up, int n_occ_dn, const double* eps_up,
                                 const double* eps_dn, const double* C_up, const double* C_dn,
                                 const double* h_core);

/* Stages (a)-(c) for the current orbitals.  omega[n_ov] receives Omega_s
 * ascending (may be NULL).  xpy[n_ov][n_ov] receives (X+Y)_ts (row t, column s)
 * with each column's largest-magnitude entry of Z made positive; it needs
 * MOLGW_FLAG_FULL_XPY (else MOLGW_E_ARG) and may be NULL.  mol = -1 runs every
 * molecule that has RI factors and orbitals (omega and xpy must then be NULL). */
int molgw_b200_rpa(molgw_ctx ctx, int mol, double* omega, double* xpy);

/* Stages (a)-(e), reusing (a)-(c) when still valid for the current orbitals.
 * sigma_x[n_basis][n_basis] and sigma_c[n_basis][n_basis] (the Hermitised qsGW
 * correlation matrix, or the qsMP2 one with MOLGW_FLAG_QSMP2) are in the basis
 * of the current MOs; either may be NULL.
 * mol = -1: every ready molecule, outputs must be NULL. */
int molgw_b200_sigma(molgw_ctx ctx, int mol, double* sigma_x, double* sigma_c);

/* One qsGW (with MOLGW_FLAG_QSMP2: qsMP2) iteration: stages (a)-(f).  The updated energies and orbitals become
 * the current ones; eps_out[n_basis] and C_out[n_basis][n_basis] receive them
 * (either may be NULL).  Occupations follow the aufbau order of eps'.
 * mol = -1: every ready molecule, outputs must be NULL. */
int molgw_b200_qs_step(molgw_ctx ctx, int mol, double* eps_out, double* C_out);

/* One-shot G0W0 (Sec. II.C: the conventional method keeps only the diagonal
 * m = n of Eq. (Sigma.c.GW)) from the current orbitals, which stay current:
 * stages (a)-(d) (reusing (a)-(c) when valid; the residues w in float64 at every
 * precision), then for every p
 *   Sigma_c,pp(eps_p) = sum_{m,s} (w^s_pm)^2 Re 1/(eps_p - eps_m +/- Omega_s -/+ i eta),
 *   Z_p = 1 / (1 - dSigma_c,pp/domega (eps_p)),
 *   eps^QP_p = eps_p + Z_p [Sigma_x,pp + Sigma_c,pp(eps_p) - v_pp],
 * v = diag(eps) - h_MO - J the potential of the input mean field (0 net with
 * Sigma_x for an input read as HF).  The quasiparticle equation is solved to
 * first order around eps_p (the paper does not name the solver).  Outputs
 * eps_qp[n_basis], z[n_basis], sigma_c_diag[n_basis] may each be NULL; mol = -1
 * runs every ready molecule (outputs NULL; fetch MOLGW_ITEM_EPS_QP etc.).
 * MOLGW_E_STATE with MOLGW_FLAG_QSMP2.  MOLGW_E_NOMEM if 2 n_basis x (blocks of m)
 * exceeds the 16 M-double split-K scratch. */
int molgw_b200_g0w0(molgw_ctx ctx, int mol, double* eps_qp, double* z, double* sigma_c_diag);

/* molgw_b200_g0w0 for the state window p_begin <= p < p_end only (the paper's
 * window of states whose self-energy is computed): the residues w^s_pm are formed
 * for those rows p alone, so their cost scales with p_end - p_begin.  Outputs have
 * p_end - p_begin entries; in the fetch items (length n_basis) only the window is
 * updated (entries that no window has computed since set_orbitals are NaN).  0 <= p_begin < p_end <= n_basis (else MOLGW_E_ARG); with mol = -1 the
 * window is clipped to each molecule's n_basis. */
int molgw_b200_g0w0_window(molgw_ctx ctx, int mol, int p_begin, int p_end, double* eps_qp, double* z,
                           double* sigma_c_diag);

/* Synchronise the context stream and return the latched device status (then
 * cleared). */
int molgw_b200_sync(molgw_ctx ctx);

/* Test hook for the error paths: latches `code` (MOLGW_E_TIMEOUT, MOLGW_E_NOCONV or
 * MOLGW_E_NUMERIC, the codes device-side checks raise) into the context's status
 * word from a one-thread kernel on the context stream, as a bounded wait that ran
 * out would; the next synchronising call returns it and clears it.  No device fault
 * is made and no kernel is stopped.  MOLGW_E_ARG for any other code. */
int molgw_b200_inject_fault(molgw_ctx ctx, int code);

/* Test hook for the bounded device waits: a grid barrier of the tridiagonalisation's
 * persistent panel kernel gives up after `grid_spins` polls (default 2^24, about 1 s)
 * with MOLGW_E_TIMEOUT, raising an abort flag on which every CTA of the launch leaves;
 * the float64 bisection of an eigenvalue stops after `bisect_rounds` rounds (default
 * and maximum 128) with MOLGW_E_NOCONV.  A negative value restores the default.  With
 * lowered bounds the results of the pass are not meaningful; the latched code reaches
 * the caller as for any device-found error, and once the defaults are back the
 * context computes as before (every launch clears its barrier block).  No fault is
 * made and no wait is endless.  MOLGW_E_ARG for a NULL context. */
int molgw_b200_set_wait_limits(molgw_ctx ctx, long long grid_spins, int bisect_rounds);

/* The symmetric matrix-vector product y = A22 v of the tridiagonalisation's panel
 * kernel (Sec. II.E's diagonalisation of the Casida matrix; LAPACK dlatrd's level-2
 * step) with MOLGW_FLAG_EIG_TC, on the context stream:
 *   MOLGW_MATVEC_AUTO  the default: the integer one;
 *   MOLGW_MATVEC_FP64  float64 arithmetic (as without MOLGW_FLAG_EIG_TC);
 *   MOLGW_MATVEC_TC    tensor cores: tile images of 7 BF16 digits (56-bit fixed point per
 *                      64 x 64 tile), exact digit-pair sums, from trailing order 1024;
 *   MOLGW_MATVEC_INT   32 x 32 -> 64-bit integer multiply-adds on 53-bit fixed-point images
 *                      (one grid per 64 x 64 tile of A22, one for v), exact products and
 *                      sums, one rounding per row, from trailing order 256.
 * The fixed-point forms are float64-accurate in the normwise sense (every value to 2^-54
 * of its group's largest), not float64 arithmetic.  Lanes of a batch (mol = -1 over
 * several molecules) always use float64.  MOLGW_E_ARG for a NULL context or another kind. */
enum molgw_matvec { MOLGW_MATVEC_AUTO = 0, MOLGW_MATVEC_FP64 = 1, MOLGW_MATVEC_TC = 2, MOLGW_MATVEC_INT = 3 };
int molgw_b200_set_panel_matvec(molgw_ctx ctx, int kind);

/* Copy an intermediate of the last pass of molecule `mol` into out[count]
 * (count must equal the item's size).  Items: */
enum molgw_item {
  MOLGW_ITEM_B = 0,        /* B[P][p][q], n_aux*n_basis^2, current orbitals           */
  MOLGW_ITEM_OMEGA = 1,    /* Omega_s, n_ov                                           */
  MOLGW_ITEM_R = 2,        /* R[P][s] = sum_t B^P_t (X+Y)_ts, n_aux*n_ov              */
  MOLGW_ITEM_SIGMA_X = 3,  /* n_basis^2                                               */
  MOLGW_ITEM_SIGMA_C = 4,  /* n_basis^2                                               */
  MOLGW_ITEM_J = 5,        /* Hartree J_pq, n_basis^2                                 */
  MOLGW_ITEM_H_MO = 6,     /* one-body h in the basis of the current MOs, n_basis^2    */
  MOLGW_ITEM_EPS = 7,      /* current eps, n_basis                                    */
  MOLGW_ITEM_C = 8,        /* current C, n_basis^2                                    */
  MOLGW_ITEM_EPS_QP = 9,   /* last molgw_b200_g0w0: eps^QP_p, n_basis                  */
  MOLGW_ITEM_Z = 10,       /* last molgw_b200_g0w0: Z_p, n_basis                       */
  MOLGW_ITEM_SIGMA_C_DIAG = 11  /* last molgw_b200_g0w0: Re Sigma_c,pp(eps_p), n_basis  */
};
int molgw_b200_fetch(molgw_ctx ctx, int mol, int item, double* out, size_t count);

/* Stages (a)-(b) only: the Casida matrix M[t][u] (n_ov x n_ov, both triangles)
 * of molecule `mol` for its current orbitals. */
int molgw_b200_rpa_matrix(molgw_ctx ctx, int mol, double* M);

/* The float64 symmetric eigensolver used by stages (c) and (f), on its own:
 * A[n][n] symmetric (read only), w[n] eigenvalues ascending, Z[n][n] (row i,
 * column k = eigenvector k, largest-magnitude entry positive; may be NULL).
 * Householder tridiagonalisation, bisection, twisted-factorisation vectors and
 * the blocked back-transformation, all on the device. */
int molgw_b200_eigh(molgw_ctx ctx, int n, const double* A, double* w, double* Z);

/* Largest n accepted by molgw_b200_eigh_noalloc. */
#define MOLGW_NOALLOC_NMAX 256

/* Allocation-free variant of molgw_b200_eigh, for callers that cannot allocate
 * device memory when they need the decomposition (an application whose own pool
 * allocator owns all device memory, a latency-bound loop that cannot pay for
 * cudaMalloc or the device-wide synchronisation of cudaFree, a plug-in running
 * after the host program has claimed its memory).  The paper has no counterpart:
 * it is a service of this library.
 *   n <= MOLGW_NOALLOC_NMAX; A[n][n] symmetric, w[n], Z[n][n] (may be NULL) are
 *   DEVICE (or managed) pointers of the current device (host memory, or memory of
 *   another device: MOLGW_E_ARG); results as for molgw_b200_eigh.  stream: the
 *   cudaStream_t to run on (NULL = legacy default).
 *   All workspace is one fixed device array of 634,042 doubles (5.07 MB) inside
 *   the library, held by every GPU that loads it until the process exits; no call
 *   allocates or frees.  The first call on a device (and the first after its
 *   context was replaced, e.g. by cudaDeviceReset) looks up that array's address
 *   with the device current, so make it before any stream capture.
 *   The call synchronises `stream` and returns the device status.
 *   Every call shares the one array: calls that overlap on the GPU (other
 *   streams, other host threads) race and must be serialised by the caller. */
int molgw_b200_eigh_noalloc(int n, const double* A, double* w, double* Z, void* stream);

/* Kernel timing collected while MOLGW_FLAG_KTIMING is set: for kernel class k
 * (enum molgw_kernel) the number of launches and their summed event time in ms
 * since the last reset.  names may be NULL.  Synchronises.  reset != 0 clears. */
enum molgw_kernel {
  MOLGW_K_GEMM_F64 = 0, MOLGW_K_TRIDIAG_PANEL = 1, MOLGW_K_TRIDIAG_SYR2K = 2,
  MOLGW_K_BISECT = 3, MOLGW_K_TWISTED = 4, MOLGW_K_BACKTRANSFORM = 5,
  MOLGW_K_SIGMA = 6, MOLGW_K_GEMM_TC = 7, MOLGW_K_MISC = 8, MOLGW_K_COUNT = 9
};
int molgw_b200_kernel_stats(molgw_ctx ctx, int64_t* launches, double* ms, int reset);

/* Choose which kernel classes are timed with events (bit k = enum molgw_kernel
 * k; 0 turns timing off, MOLGW_FLAG_KTIMING at create time sets all bits).
 * Synchronises and returns the latched device status. */
int molgw_b200_set_timing(molgw_ctx ctx, uint32_t class_mask);

/* Number of device kernels this context has launched since creation (a graph
 * replay counts the kernels the graph holds). */
int64_t molgw_b200_launch_count(molgw_ctx ctx);

/* Library extension (the paper has no counterpart): a tensor-core GEMM on its
 * own, C[m][n] = sum_k A[m][k] B[n][k] for row-major float64 A[M][K], B[N][K],
 * C[M][N] (host or device memory), so that the tensor-core arithmetic can be
 * checked against float64.  digits = 0: the split of the context's precision
 * (not MOLGW_PREC_FP64, else MOLGW_E_ARG); digits = 4 or 7: the fixed-point
 * engine with that many digits (any precision).  Allocates temporaries and
 * synchronises. */
int molgw_b200_tc_gemm(molgw_ctx ctx, int digits, int M, int N, int K, const double* A, const double* B, double* C);

/* Library extension (the paper has no counterpart): tune the schedule.
 * Runs trial qs_steps of all ready molecules (mol = -1) and puts every
 * molecule's energies, orbitals and h_MO back after each: a first trial times
 * every float64 GEMM shape of the pass with each tile side (64, 48, 40, 32;
 * the results are bit-identical, only the time differs) and keeps the fastest
 * per shape; then one trial each with 4, 8, 12 and 16 concurrent lanes (fewer
 * with fewer molecules) picks the lane count used by later mol = -1 calls when
 * opts.lanes is 0.  *lanes_out (may be NULL) receives it.  Synchronises;
 * allocates a snapshot of the orbitals meanwhile.  MOLGW_E_STATE when no
 * molecule is ready. */
int molgw_b200_autotune(molgw_ctx ctx, int32_t* lanes_out);

/* Lane count the next mol = -1 call uses. */
int32_t molgw_b200_lanes(molgw_ctx ctx);

/* The lane plan of a batch (mol = -1), computed on the host with no context and no
 * device: molecule k of n_mols goes to lane lane_of[k] and is issued there in position
 * slot[k] (slot may be NULL).  A pass's relative cost is n_ov^3 (eigensolve) plus
 * 2 nb^2 n_ov na per spin channel (residues); with MOLGW_FLAG_QSMP2 in flags it is
 * 4 nb^2 n_ov na + 2 nb^3 n_ov.  Molecules are taken in order of decreasing cost (equal
 * costs by index), each to the lane with the least cost so far (equal: the lowest
 * lane), over max(1, min(lanes, n_mols)) lanes; lanes = 0 means the default of 8, and
 * at most 16 are used.  A context whose opts.lanes equals `lanes` (and which was not
 * autotuned) runs the same plan.  n_basis, n_aux, n_occ_up: [n_mols]; n_occ_dn: NULL
 * for closed shells (n_occ_up is then n_occ), else [n_mols] with -1 for a closed shell.
 * Returns the number of lanes used, or MOLGW_E_ARG for sizes that set_ri or
 * set_orbitals(_open) would refuse (and for open shells with MOLGW_FLAG_QSMP2). */
int molgw_b200_plan_batch(int n_mols, const int32_t* n_basis, const int32_t* n_aux, const int32_t* n_occ_up,
                          const int32_t* n_occ_dn, uint32_t flags, int lanes, int32_t* lane_of, int32_t* slot);

/* Library extension (the paper has no counterpart): number of qs_step calls
 * served by replaying a captured graph (MOLGW_FLAG_GRAPH); -1 once a capture
 * failed and the context went back to issuing the launches one by one. */
int64_t molgw_b200_graph_replays(molgw_ctx ctx);

/* Free every resource of the context (synchronises first).  Returns the
 * latched device status.  ctx may be NULL. */
int molgw_b200_destroy(molgw_ctx ctx);

/* Static text for a status code. */
const char* molgw_b200_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* MOLGW_GB300_H */
