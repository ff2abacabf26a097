// C ABI of the RI-qsGW library: context, per-molecule state machine, copies.
#include <string.h>

#include <new>

#include "stages.cuh"

using namespace molgw;

struct molgw_ctx_s {
  molgw_opts opts{};
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int* d_status = nullptr;
  int* h_status = nullptr;   // pinned mirror
  KTimer timer;
  Exec ex;
  std::vector<MolBuf> mols;
  std::vector<TcBufs> tcb;   // split operands of the tensor-core path (precision != FP64)
  Scratch scr;
  EigWork eig;
  int eig_n = 0, eig_cols = 0;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MOLGW_OK;
  if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return MOLGW_E_NOMEM; }
  return MOLGW_E_CUDA;
}

int launch_status() { return cuda_status(cudaGetLastError()); }

double* dalloc(std::vector<void*>& v, size_t n_doubles, int* err) {
  void* p = nullptr;
  if (*err) return nullptr;
  if (cudaMalloc(&p, std::max<size_t>(n_doubles, 1) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    *err = MOLGW_E_NOMEM;
    return nullptr;
  }
  v.push_back(p);
  return (double*)p;
}

void free_all(std::vector<void*>& v) {
  for (void* p : v) cudaFree(p);
  v.clear();
}

int copy_in(molgw_ctx c, double* dst, const double* src, size_t n) {
  return cuda_status(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, c->st));
}

// Copy n doubles out; sets *need_sync when dst is host memory.
int copy_out(molgw_ctx c, double* dst, const double* src, size_t n, bool* need_sync) {
  if (!is_device_ptr(dst)) *need_sync = true;
  return cuda_status(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, c->st));
}

int read_status(molgw_ctx c) {
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return MOLGW_E_CUDA;
  e = cudaMemcpy(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return MOLGW_E_CUDA;
  const int s = *c->h_status;
  if (s != 0) cudaMemset(c->d_status, 0, sizeof(int));
  c->timer.resolve();
  return s;
}

bool use_tc_ctx(molgw_ctx c) { return c->opts.precision != MOLGW_PREC_FP64; }

int ensure_eig(molgw_ctx c, int n, int ncols) {
  if (n <= c->eig_n && ncols <= c->eig_cols) return MOLGW_OK;
  const int nn = std::max(n, c->eig_n), nc = std::max(ncols, c->eig_cols);
  cudaStreamSynchronize(c->st);
  int r = eig_work_alloc(c->eig, nn, nc);
  if (r) { c->eig_n = c->eig_cols = 0; return r; }
  c->eig_n = nn; c->eig_cols = nc;
  return MOLGW_OK;
}

// Packed residue buffers of the float64 path, when the device has room for them
// (they halve the residue flops); otherwise the blocked route without them is used.
void ensure_packed(molgw_ctx c, int nb, int na, long long nov) {
  Scratch& s = c->scr;
  const size_t npair = (size_t)nb * (nb + 1) / 2;
  const size_t want_w = npair * nov, want_b = npair * na;
  if (want_w <= s.wpk_cap && want_b <= s.bpt_cap) return;
  cudaStreamSynchronize(c->st);
  if (s.pk_base) cudaFree(s.pk_base);
  s.pk_base = nullptr; s.wpk = s.bpt = nullptr; s.wpk_cap = s.bpt_cap = 0;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); return; }
  const size_t bytes = (want_w + want_b) * sizeof(double);
  if (bytes > fr / 3) return;
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return; }
  s.pk_base = p;
  s.wpk = (double*)p;
  s.bpt = s.wpk + want_w;
  s.wpk_cap = want_w;
  s.bpt_cap = want_b;
}

int ensure_scratch(molgw_ctx c, int nb, int na, long long nov) {
  Scratch& s = c->scr;
  const size_t want_w = std::max<size_t>((size_t)nb * nov,
                                         std::min<size_t>((size_t)nb * nb * nov, (size_t)48 << 20));
  if (!use_tc_ctx(c)) ensure_packed(c, nb, na, nov);
  if (nb <= s.nb_cap && na <= s.na_cap && want_w <= s.wblk_cap) return MOLGW_OK;
  cudaStreamSynchronize(c->st);
  const int nbc = std::max(nb, s.nb_cap), nac = std::max(na, s.na_cap);
  const size_t wc = std::max(want_w, s.wblk_cap);
  const size_t skc = (size_t)16 << 20;
  if (s.base) cudaFree(s.base);
  void* pk = s.pk_base; double* wpk = s.wpk; double* bpt = s.bpt;
  const size_t wcap = s.wpk_cap, bcap = s.bpt_cap;
  s = Scratch{};
  s.pk_base = pk; s.wpk = wpk; s.bpt = bpt; s.wpk_cap = wcap; s.bpt_cap = bcap;
  const size_t nn = (size_t)nbc * nbc;
  const size_t total = nac + skc + 2 * wc + 3 * nn;
  void* p = nullptr;
  if (cudaMalloc(&p, total * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return MOLGW_E_NOMEM; }
  double* q = (double*)p;
  s.base = p;
  s.rho = q; q += nac;
  s.splitk = q; s.splitk_cap = skc; q += skc;
  s.wblk = q; q += wc;
  s.pblk = q; q += wc;
  s.wblk_cap = wc;
  s.S = q; q += nn; s.H = q; q += nn; s.U = q; q += nn;
  s.nb_cap = nbc; s.na_cap = nac;
  return MOLGW_OK;
}

bool mol_ok(molgw_ctx c, int mol) { return c && mol >= 0 && mol < (int)c->mols.size(); }

bool use_tc(molgw_ctx c) { return c->opts.precision != MOLGW_PREC_FP64; }
int tc_prec(molgw_ctx c) {
  if (c->opts.precision == MOLGW_PREC_TF32X3) return TC_TF32X3;
  if (c->opts.precision == MOLGW_PREC_BF16X6) return TC_BF16X6;
  return TC_BF16X3;
}

// m values per self-energy block: w and g*w (hi and lo each) within about 1 GB
int tc_mblock(int prec, int nb, long long nov) {
  const long long per_m = 2LL * tc_slices(prec) * nb * tc_pad(nov, prec) * tc_elem_bytes(prec);
  return (int)std::max<long long>(1, std::min<long long>(nb, (1LL << 30) / std::max<long long>(per_m, 1)));
}

// Run the pass of one molecule up to a stage: 'b' (M), 'c' (rpa), 'e' (sigma), 'f' (qs step).
int run_pass(molgw_ctx c, int mol, char upto) {
  MolBuf& m = c->mols[mol];
  if (!m.have_ri || !m.have_orb) return MOLGW_E_STATE;
  const bool full = (c->opts.flags & MOLGW_FLAG_FULL_XPY) != 0;
  int r = ensure_scratch(c, m.nb, m.na, m.nov);
  if (!r) r = ensure_eig(c, (int)std::max<long long>(m.nov, m.nb),
                         std::max<int>(std::max(m.na, m.nb), full ? (int)m.nov : 0));
  if (r) return r;
  Exec& ex = c->ex;
  const bool tc = use_tc(c);
  const bool tc_ab = tc && (c->opts.flags & MOLGW_FLAG_TC_AB);
  TcBufs& tb = c->tcb[mol];
  if (!m.b_valid) {
    if (tc_ab) {
      r = stage_ri_mo_transform_tc(ex, m, tb);
      if (r) return r;
    } else {
      stage_ri_mo_transform(ex, m);
    }
    m.b_valid = m.have_b = true;
  }
  if (!m.h_ready) {
    stage_j_sigx(ex, m, c->scr);
    derive_h_from_hf(ex, m);
    m.jx_valid = m.have_jx = true;
    m.h_ready = true;
  }
  if (upto == 'b') {
    if (tc_ab) {
      r = stage_rpa_build_tc(ex, m, tb);
      if (r) return r;
    } else {
      stage_rpa_build(ex, m);
    }
    m.rpa_valid = false;
    return launch_status();
  }
  if (!m.rpa_valid) {
    if (tc_ab) {
      r = stage_rpa_build_tc(ex, m, tb);
      if (r) return r;
    } else {
      stage_rpa_build(ex, m);
    }
    stage_rpa_eigensolve(ex, m, c->eig, c->scr, full);
    m.rpa_valid = m.have_rpa = true;
  }
  if (upto >= 'e' && !m.sigma_valid) {
    if (!m.jx_valid) {
      stage_j_sigx(ex, m, c->scr);
      m.jx_valid = m.have_jx = true;
    }
    if (tc) {
      r = stage_sigma_tc(ex, m, tb, c->scr, c->opts.eta);
      if (r) return r;
    } else {
      stage_sigma(ex, m, c->scr, c->opts.eta);
    }
    m.sigma_valid = m.have_sigma = true;
  }
  if (upto == 'f') {
    stage_qs_update(ex, m, c->eig, c->scr);
    m.b_valid = m.jx_valid = m.rpa_valid = m.sigma_valid = false;
  }
  return launch_status();
}

bool ready(const MolBuf& m) { return m.have_ri && m.have_orb; }

}  // namespace

extern "C" {

int molgw_b200_create(const molgw_opts* o, molgw_ctx* out) {
  if (!out) return MOLGW_E_ARG;
  *out = nullptr;
  if (!o || o->struct_size != (int32_t)sizeof(molgw_opts)) return MOLGW_E_ARG;
  if (o->precision < MOLGW_PREC_FP64 || o->precision > MOLGW_PREC_BF16X6) return MOLGW_E_ARG;
  if (o->max_mols < 1 || !(o->eta > 0.0)) return MOLGW_E_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) { cudaGetLastError(); return MOLGW_E_CUDA; }
  if (o->device < 0 || o->device >= ndev) return MOLGW_E_ARG;
  molgw_ctx c = new (std::nothrow) molgw_ctx_s();
  if (!c) return MOLGW_E_NOMEM;
  c->opts = *o;
  c->device = o->device;
  DeviceGuard g(c->device);
  if (o->stream || (o->flags & MOLGW_FLAG_USE_STREAM)) {
    c->st = (cudaStream_t)o->stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) { delete c; return MOLGW_E_CUDA; }
    c->own_stream = true;
  }
  if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->h_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (c->d_status) cudaFree(c->d_status);
    if (c->own_stream) cudaStreamDestroy(c->st);
    delete c;
    return MOLGW_E_NOMEM;
  }
  cudaMemsetAsync(c->d_status, 0, sizeof(int), c->st);
  c->mols.resize(o->max_mols);
  c->tcb.resize(o->max_mols);
  c->timer.enabled = (o->flags & MOLGW_FLAG_KTIMING) != 0;
  c->timer.mask = c->timer.enabled ? 0xffffffffu : 0u;
  c->ex.st = c->st;
  c->ex.status = c->d_status;
  c->ex.timer = &c->timer;
  *out = c;
  return MOLGW_OK;
}

int molgw_b200_set_ri(molgw_ctx c, int mol, int n_basis, int n_aux, const double* L) {
  if (!mol_ok(c, mol) || !L || n_basis < 2 || n_aux < 1) return MOLGW_E_ARG;
  if ((long long)n_aux * n_basis * n_basis > (1LL << 40)) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  MolBuf& m = c->mols[mol];
  const size_t nl = (size_t)n_aux * n_basis * n_basis;
  m.have_ri = m.have_orb = false;
  m.b_valid = m.jx_valid = m.rpa_valid = m.sigma_valid = false;
  m.have_b = m.have_rpa = m.have_jx = m.have_sigma = false;
  m.h_ready = false;
  if (m.ri_allocs.empty() || m.nb != n_basis || m.na != n_aux) {
    cudaStreamSynchronize(c->st);
    free_all(m.ri_allocs);
    free_all(m.orb_allocs);   // orbital-size buffers depend on n_basis and n_aux
    m.eps = nullptr;
    m.alloc_no = 0;
    m.nb = n_basis; m.na = n_aux;
    int err = 0;
    m.L = dalloc(m.ri_allocs, nl, &err);
    m.B = dalloc(m.ri_allocs, nl, &err);
    m.T1 = dalloc(m.ri_allocs, nl, &err);
    TcBufs& tb = c->tcb[mol];
    free_all(tb.ri_allocs);
    free_all(tb.orb_allocs);
    if (use_tc(c) && (c->opts.flags & MOLGW_FLAG_TC_AB)) {
      double* base = dalloc(tb.ri_allocs, tc_ri_doubles(tc_prec(c), n_basis, n_aux), &err);
      if (!err) tc_ri_carve(tb, tc_prec(c), n_basis, n_aux, base);
    }
    if (err) { free_all(m.ri_allocs); free_all(tb.ri_allocs); m.nb = m.na = 0; return err; }
  }
  int r = copy_in(c, m.L, L, nl);
  if (r) return r;
  check_finite(c->ex, m.L, (long long)nl);
  if (use_tc(c) && (c->opts.flags & MOLGW_FLAG_TC_AB)) tc_split_ri(c->ex, m, c->tcb[mol]);
  m.have_ri = true;
  return launch_status();
}

int molgw_b200_set_orbitals(molgw_ctx c, int mol, int n_occ, const double* eps, const double* C,
                            const double* h_core) {
  if (!mol_ok(c, mol) || !eps || !C) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  MolBuf& m = c->mols[mol];
  if (!m.have_ri) return MOLGW_E_STATE;
  const int nb = m.nb, na = m.na;
  if (n_occ < 1 || n_occ >= nb) return MOLGW_E_ARG;
  const long long nov = (long long)n_occ * (nb - n_occ);
  const bool full = (c->opts.flags & MOLGW_FLAG_FULL_XPY) != 0;
  if (m.orb_allocs.empty() || m.alloc_no != n_occ) {
    cudaStreamSynchronize(c->st);
    free_all(m.orb_allocs);
    m.have_orb = false;
    int err = 0;
    const size_t nn = (size_t)nb * nb;
    m.eps = dalloc(m.orb_allocs, nb, &err);
    m.C = dalloc(m.orb_allocs, nn, &err);
    m.hmo = dalloc(m.orb_allocs, nn, &err);
    m.J = dalloc(m.orb_allocs, nn, &err);
    m.sigx = dalloc(m.orb_allocs, nn, &err);
    m.sigc = dalloc(m.orb_allocs, nn, &err);
    m.D = dalloc(m.orb_allocs, nov, &err);
    m.Om = dalloc(m.orb_allocs, nov, &err);
    m.Xv = dalloc(m.orb_allocs, (size_t)nov * na, &err);
    m.R = dalloc(m.orb_allocs, (size_t)nov * na, &err);
    m.M = dalloc(m.orb_allocs, (size_t)nov * nov, &err);
    m.ZT = dalloc(m.orb_allocs, (size_t)nov * nov, &err);
    m.XpY = full ? dalloc(m.orb_allocs, (size_t)nov * nov, &err) : nullptr;
    TcBufs& tb = c->tcb[mol];
    free_all(tb.orb_allocs);
    if (use_tc(c) && !err) {
      const int prec = tc_prec(c);
      const int mb = tc_mblock(prec, nb, nov);
      const size_t nd = tc_orb_doubles(prec, nb, na, nov, mb, tc_pad(nov, prec));
      double* base = dalloc(tb.orb_allocs, nd, &err);
      if (!err) {
        // padding columns that no kernel writes (X beyond nb, w and g*w beyond n_ov) must read as zero
        cudaMemsetAsync(base, 0, nd * sizeof(double), c->st);
        tc_bufs_carve(tb, prec, nb, na, nov, mb, base);
      }
    }
    if (err) { free_all(m.orb_allocs); free_all(tb.orb_allocs); m.eps = nullptr; m.alloc_no = 0; return err; }
    m.alloc_no = n_occ;
  }
  m.no = n_occ;
  m.nov = nov;
  int r = copy_in(c, m.eps, eps, nb);
  if (!r) r = copy_in(c, m.C, C, (size_t)nb * nb);
  if (r) return r;
  check_finite(c->ex, m.eps, nb);
  check_finite(c->ex, m.C, (long long)nb * nb);
  m.have_orb = true;
  m.b_valid = m.jx_valid = m.rpa_valid = m.sigma_valid = false;
  m.have_b = m.have_rpa = m.have_jx = m.have_sigma = false;
  m.h_ready = false;
  if (h_core) {
    r = ensure_scratch(c, nb, na, nov);
    if (r) return r;
    // stage h_AO in the T1 buffer (n_aux*nb*nb >= nb*nb), then h_MO = C^T h C
    r = copy_in(c, m.T1, h_core, (size_t)nb * nb);
    if (r) return r;
    h_ao_to_mo(c->ex, m, m.T1, c->scr);
    m.h_ready = true;
  }
  return launch_status();
}

static int for_each_ready(molgw_ctx c, char upto) {
  int any = 0;
  for (int k = 0; k < (int)c->mols.size(); ++k) {
    if (!ready(c->mols[k])) continue;
    any = 1;
    int r = run_pass(c, k, upto);
    if (r) return r;
  }
  return any ? MOLGW_OK : MOLGW_E_STATE;
}

int molgw_b200_rpa(molgw_ctx c, int mol, double* omega, double* xpy) {
  if (!c) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  if (mol == -1) {
    if (omega || xpy) return MOLGW_E_ARG;
    return for_each_ready(c, 'c');
  }
  if (!mol_ok(c, mol)) return MOLGW_E_ARG;
  if (xpy && !(c->opts.flags & MOLGW_FLAG_FULL_XPY)) return MOLGW_E_ARG;
  MolBuf& m = c->mols[mol];
  if (!ready(m)) return MOLGW_E_STATE;
  int r = run_pass(c, mol, 'c');
  if (r) return r;
  bool sync = false;
  if (omega) r = copy_out(c, omega, m.Om, m.nov, &sync);
  if (!r && xpy) r = copy_out(c, xpy, m.XpY, (size_t)m.nov * m.nov, &sync);
  if (r) return r;
  return sync ? read_status(c) : MOLGW_OK;
}

int molgw_b200_sigma(molgw_ctx c, int mol, double* sigma_x, double* sigma_c) {
  if (!c) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  if (mol == -1) {
    if (sigma_x || sigma_c) return MOLGW_E_ARG;
    return for_each_ready(c, 'e');
  }
  if (!mol_ok(c, mol)) return MOLGW_E_ARG;
  MolBuf& m = c->mols[mol];
  if (!ready(m)) return MOLGW_E_STATE;
  int r = run_pass(c, mol, 'e');
  if (r) return r;
  bool sync = false;
  const size_t nn = (size_t)m.nb * m.nb;
  if (sigma_x) r = copy_out(c, sigma_x, m.sigx, nn, &sync);
  if (!r && sigma_c) r = copy_out(c, sigma_c, m.sigc, nn, &sync);
  if (r) return r;
  return sync ? read_status(c) : MOLGW_OK;
}

int molgw_b200_qs_step(molgw_ctx c, int mol, double* eps_out, double* C_out) {
  if (!c) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  if (mol == -1) {
    if (eps_out || C_out) return MOLGW_E_ARG;
    return for_each_ready(c, 'f');
  }
  if (!mol_ok(c, mol)) return MOLGW_E_ARG;
  MolBuf& m = c->mols[mol];
  if (!ready(m)) return MOLGW_E_STATE;
  int r = run_pass(c, mol, 'f');
  if (r) return r;
  bool sync = false;
  if (eps_out) r = copy_out(c, eps_out, m.eps, m.nb, &sync);
  if (!r && C_out) r = copy_out(c, C_out, m.C, (size_t)m.nb * m.nb, &sync);
  if (r) return r;
  return sync ? read_status(c) : MOLGW_OK;
}

int molgw_b200_sync(molgw_ctx c) {
  if (!c) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  return read_status(c);
}

int molgw_b200_fetch(molgw_ctx c, int mol, int item, double* out, size_t count) {
  if (!mol_ok(c, mol) || !out) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  MolBuf& m = c->mols[mol];
  const size_t nn = (size_t)m.nb * m.nb;
  const double* src = nullptr;
  size_t n = 0;
  bool avail = false;
  switch (item) {
    case MOLGW_ITEM_B: src = m.B; n = (size_t)m.na * nn; avail = m.have_b; break;
    case MOLGW_ITEM_OMEGA: src = m.Om; n = m.nov; avail = m.have_rpa; break;
    case MOLGW_ITEM_R: src = m.R; n = (size_t)m.na * m.nov; avail = m.have_rpa; break;
    case MOLGW_ITEM_SIGMA_X: src = m.sigx; n = nn; avail = m.have_jx; break;
    case MOLGW_ITEM_SIGMA_C: src = m.sigc; n = nn; avail = m.have_sigma; break;
    case MOLGW_ITEM_J: src = m.J; n = nn; avail = m.have_jx; break;
    case MOLGW_ITEM_H_MO: src = m.hmo; n = nn; avail = m.h_ready; break;
    case MOLGW_ITEM_EPS: src = m.eps; n = m.nb; avail = m.have_orb; break;
    case MOLGW_ITEM_C: src = m.C; n = nn; avail = m.have_orb; break;
    default: return MOLGW_E_ARG;
  }
  if (!avail) return MOLGW_E_STATE;
  if (count != n) return MOLGW_E_ARG;
  bool sync = false;
  int r = copy_out(c, out, src, n, &sync);
  if (r) return r;
  return sync ? read_status(c) : MOLGW_OK;
}

int molgw_b200_rpa_matrix(molgw_ctx c, int mol, double* M) {
  if (!mol_ok(c, mol) || !M) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  MolBuf& m = c->mols[mol];
  if (!ready(m)) return MOLGW_E_STATE;
  int r = run_pass(c, mol, 'b');
  if (r) return r;
  // the build keeps the lower 64x64 tiles and full diagonal tiles: mirror them
  fill_upper(c->ex, m.M, m.nov);
  bool sync = false;
  r = copy_out(c, M, m.M, (size_t)m.nov * m.nov, &sync);
  if (r) return r;
  return sync ? read_status(c) : MOLGW_OK;
}

int molgw_b200_eigh(molgw_ctx c, int n, const double* A, double* w, double* Z) {
  if (!c || n < 1 || !A || !w) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  int r = ensure_eig(c, n, n);
  if (r) return r;
  std::vector<void*> tmp;
  int err = 0;
  double* dA = dalloc(tmp, (size_t)n * n, &err);
  double* dZ = Z ? dalloc(tmp, (size_t)n * n, &err) : nullptr;
  if (err) { free_all(tmp); return err; }
  r = copy_in(c, dA, A, (size_t)n * n);
  if (!r) {
    eigh_dense(c->ex, c->eig, n, dA, dZ);
    r = launch_status();
  }
  bool sync = false;
  if (!r) r = copy_out(c, w, c->eig.lam, n, &sync);
  if (!r && Z) r = copy_out(c, Z, dZ, (size_t)n * n, &sync);
  int s = read_status(c);   // the temporaries are freed below: always synchronise
  free_all(tmp);
  return r ? r : s;
}

int molgw_b200_kernel_stats(molgw_ctx c, int64_t* launches, double* ms, int reset) {
  if (!c) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  int s = read_status(c);
  for (int k = 0; k < MOLGW_K_COUNT; ++k) {
    if (launches) launches[k] = c->timer.launches[k];
    if (ms) ms[k] = c->timer.ms[k];
  }
  if (reset) {
    for (int k = 0; k < MOLGW_K_COUNT; ++k) { c->timer.launches[k] = 0; c->timer.ms[k] = 0.0; }
  }
  return s;
}

int64_t molgw_b200_launch_count(molgw_ctx c) { return c ? c->timer.total_launches : 0; }

int molgw_b200_set_timing(molgw_ctx c, uint32_t class_mask) {
  if (!c) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  int s = read_status(c);
  c->timer.mask = class_mask;
  c->timer.enabled = class_mask != 0;
  return s;
}

int molgw_b200_destroy(molgw_ctx c) {
  if (!c) return MOLGW_OK;
  int s;
  {
    DeviceGuard g(c->device);
    s = read_status(c);
    for (auto& m : c->mols) { free_all(m.ri_allocs); free_all(m.orb_allocs); }
    for (auto& t : c->tcb) { free_all(t.ri_allocs); free_all(t.orb_allocs); }
    if (c->scr.base) cudaFree(c->scr.base);
    if (c->scr.pk_base) cudaFree(c->scr.pk_base);
    eig_work_free(c->eig);
    cudaFree(c->d_status);
    cudaFreeHost(c->h_status);
    if (c->own_stream) cudaStreamDestroy(c->st);
  }
  delete c;
  return s;
}

const char* molgw_b200_status_string(int s) {
  switch (s) {
    case MOLGW_OK: return "ok";
    case MOLGW_E_ARG: return "bad argument";
    case MOLGW_E_STATE: return "call out of order";
    case MOLGW_E_NOMEM: return "device allocation failed";
    case MOLGW_E_CUDA: return "CUDA runtime error";
    case MOLGW_E_NOCONV: return "eigensolver iteration cap reached";
    case MOLGW_E_TIMEOUT: return "bounded device wait ran out";
    case MOLGW_E_NUMERIC: return "non-positive RPA eigenvalue or non-finite value";
    default: return "unknown status";
  }
}

}  // extern "C"
