// C ABI of the RI-qsGW library: context, per-molecule state machine, copies.
#include <string.h>

#include <new>

#include <nvtx3/nvToolsExt.h>

#include "stages.cuh"

using namespace molgw;

// One execution lane: a stream with its own scratch, eigensolver workspace and
// tensor-core operand arena.  Lane 0 runs on the context stream; a batch call
// (mol = -1) forks further lanes from it and joins them back with events.
struct Lane {
  cudaStream_t st = nullptr;
  bool own_stream = false;
  cudaEvent_t done = nullptr;
  Exec ex;
  Scratch scr;
  EigWork eig;
  int eig_n = 0, eig_cols = 0;
  TcBufs tco;                 // orbital-size split operands, carved per molecule
  FxBufs fxo;                 // the same for the fixed-point precision
  void* tco_base = nullptr;
  size_t tco_cap = 0;         // doubles
  size_t pk_fail = 0;         // packed-residue request that did not fit (not retried)
  void* eigfx = nullptr;      // MOLGW_FLAG_EIG_TC: fixed-point operands of the trailing updates
  long long eigfx_rows = 0, eigfx_cols = 0;
  void* eigsv = nullptr;      // MOLGW_FLAG_EIG_TC, lane 0: tile images of the panel mat-vec
  long long eigsv_n = 0;
};

constexpr int kMaxLanes = 16;
constexpr int kDefaultLanes = 8;

struct molgw_ctx_s {
  molgw_opts opts{};
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int* d_status = nullptr;
  int* h_status = nullptr;   // pinned mirror
  KTimer timer;
  std::vector<MolBuf> mols;
  std::vector<TcBufs> tcb;   // per molecule: split L of the tensor-core path (MOLGW_FLAG_TC_AB)
  std::vector<Lane> lanes;   // lanes[0] is the context stream
  cudaEvent_t fork = nullptr;
  uint64_t gen = 1;          // bumped whenever a buffer a captured graph may use is (re)allocated
  // captured qs_step (MOLGW_FLAG_GRAPH)
  cudaGraphExec_t gexec = nullptr;
  int graph_mol = -2;
  uint64_t graph_gen = 0;
  std::vector<char> graph_set;   // molecules the graph covers (mol = -1)
  int64_t graph_launches[MOLGW_K_COUNT] = {0};
  bool graph_off = false;        // capture failed once: run eagerly from then on
  int64_t graph_replays = 0;
  int graph_lanes = 0;           // lane count of the captured plan
  int tuned_lanes = 0;           // molgw_b200_autotune's choice (0: none)
  int g0w0_p0 = 0, g0w0_p1 = 0;  // state window of the G0W0 call in flight (clipped per molecule)
  GemmTuner tuner;               // float64 GEMM tile choices (molgw_b200_autotune)
  long long grid_spins = kGridSpinLimit;   // molgw_b200_set_wait_limits
  int bisect_rounds = kBisectRounds;
  int panel_matvec = MOLGW_MATVEC_AUTO;    // molgw_b200_set_panel_matvec
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

void free_all(std::vector<void*>& v);

// Release the spin-down channel of an open-shell molecule (if any).
void drop_open(MolBuf& m) {
  if (!m.dn) return;
  free_all(m.dn->ri_allocs);
  free_all(m.dn->orb_allocs);
  m.dn.reset();
  m.nov_up = 0;
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

// Latches a device-detected error code the way the kernels' checks do (test hook).
__global__ void k_inject_status(int* status, int code) { set_status(status, code); }

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

bool use_tc(molgw_ctx c) { return c->opts.precision != MOLGW_PREC_FP64; }
bool use_fx(molgw_ctx c) { return c->opts.precision == MOLGW_PREC_BF16X10; }
bool use_tc_ab(molgw_ctx c) { return use_tc(c) && (c->opts.flags & MOLGW_FLAG_TC_AB); }
bool use_mp2(molgw_ctx c) { return (c->opts.flags & MOLGW_FLAG_QSMP2) != 0; }
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

bool mol_ok(molgw_ctx c, int mol) { return c && mol >= 0 && mol < (int)c->mols.size(); }

// Lane k, created on first use (lane 0 is the context stream).
int lane_get(molgw_ctx c, int k, Lane** out) {
  while ((int)c->lanes.size() <= k) {
    Lane l;
    const int idx = (int)c->lanes.size();
    if (idx == 0) {
      l.st = c->st;
    } else {
      if (cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); return MOLGW_E_CUDA; }
      l.own_stream = true;
      if (cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(l.st);
        return MOLGW_E_CUDA;
      }
    }
    l.ex.st = l.st;
    l.ex.status = c->d_status;
    l.ex.timer = &c->timer;
    l.ex.tuner = &c->tuner;
    l.ex.grid_spins = c->grid_spins;
    l.ex.bisect_rounds = c->bisect_rounds;
    l.ex.panel_matvec = c->panel_matvec;
    c->lanes.push_back(l);
  }
  *out = &c->lanes[k];
  return MOLGW_OK;
}

void lane_free(Lane& l) {
  if (l.scr.base) cudaFree(l.scr.base);
  if (l.scr.pk_base) cudaFree(l.scr.pk_base);
  if (l.tco_base) cudaFree(l.tco_base);
  if (l.eigfx) cudaFree(l.eigfx);
  if (l.eigsv) cudaFree(l.eigsv);
  eig_work_free(l.eig);
  if (l.done) cudaEventDestroy(l.done);
  if (l.own_stream) cudaStreamDestroy(l.st);
}

int ensure_eig(molgw_ctx c, Lane& l, int n, int ncols) {
  if (n <= l.eig_n && ncols <= l.eig_cols) return MOLGW_OK;
  if (l.ex.capturing) return MOLGW_E_STATE;
  const int nn = std::max(n, l.eig_n), nc = std::max(ncols, l.eig_cols);
  cudaStreamSynchronize(l.st);
  ++c->gen;
  int r = eig_work_alloc(l.eig, nn, nc);
  if (r) { l.eig_n = l.eig_cols = 0; return r; }
  l.eig_n = nn; l.eig_cols = nc;
  return MOLGW_OK;
}

bool use_eig_tc(molgw_ctx c) { return (c->opts.flags & MOLGW_FLAG_EIG_TC) != 0; }

// Attach (allocating if needed) the fixed-point arena of the eigensolver's
// trailing updates to the lane's workspace (MOLGW_FLAG_EIG_TC), sized for eig_n.
int ensure_eigfx(molgw_ctx c, Lane& l) {
  if (!use_eig_tc(c)) {
    l.eig.fx = nullptr;
    l.eig.fx_rows = 0;
    l.eig.sv = nullptr;
    l.eig.sv_n = 0;
    return MOLGW_OK;
  }
  const long long rows = l.eig_n, cols = l.eig_cols;
  if (rows > l.eigfx_rows || cols > l.eigfx_cols) {
    if (l.ex.capturing) return MOLGW_E_STATE;
    cudaStreamSynchronize(l.st);
    ++c->gen;
    if (l.eigfx) cudaFree(l.eigfx);
    l.eigfx = nullptr;
    l.eigfx_rows = l.eigfx_cols = 0;
    if (cudaMalloc(&l.eigfx, eig_fx_bytes(rows, cols)) != cudaSuccess) {
      cudaGetLastError();
      l.eigfx = nullptr;
      return MOLGW_E_NOMEM;
    }
    l.eigfx_rows = rows;
    l.eigfx_cols = cols;
  }
  l.eig.fx = l.eigfx;
  l.eig.fx_rows = l.eigfx_rows;
  l.eig.fx_cols = l.eigfx_cols;
  // the tensor-core mat-vec of the panel kernel runs on the context stream only (lane 0):
  // its persistent launch holds one CTA per SM and TMEM, which concurrent lanes would share;
  // the integer mat-vec runs on every lane (with the lane's share of the SMs)
  const bool int_matvec = c->panel_matvec == MOLGW_MATVEC_AUTO || c->panel_matvec == MOLGW_MATVEC_INT;
  if (&l == &c->lanes[0] || int_matvec) {
    if (rows > l.eigsv_n) {
      if (l.ex.capturing) return MOLGW_E_STATE;
      cudaStreamSynchronize(l.st);
      ++c->gen;
      if (l.eigsv) cudaFree(l.eigsv);
      l.eigsv = nullptr;
      l.eigsv_n = 0;
      if (cudaMalloc(&l.eigsv, eig_sv_bytes(rows)) != cudaSuccess) {
        cudaGetLastError();
        l.eigsv = nullptr;
        return MOLGW_E_NOMEM;
      }
      l.eigsv_n = rows;
    }
    l.eig.sv = l.eigsv;
    l.eig.sv_n = l.eigsv_n;
  }
  return MOLGW_OK;
}

// Packed residue buffers of the float64 path, when the device has room for them
// (they halve the residue flops); otherwise the blocked route without them is used.
void ensure_packed(molgw_ctx c, Lane& l, int nb, int na, long long nov) {
  Scratch& s = l.scr;
  const size_t npair = (size_t)nb * (nb + 1) / 2;
  const size_t want_w = npair * nov, want_b = npair * na;
  if (want_w <= s.wpk_cap && want_b <= s.bpt_cap) return;
  if (l.pk_fail && want_w >= l.pk_fail) return;   // did not fit before: stay on the blocked route
  if (l.ex.capturing) return;
  cudaStreamSynchronize(l.st);
  ++c->gen;
  if (s.pk_base) cudaFree(s.pk_base);
  s.pk_base = nullptr; s.wpk = s.bpt = nullptr; s.wpk_cap = s.bpt_cap = 0;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); l.pk_fail = want_w; return; }
  const size_t bytes = (want_w + want_b) * sizeof(double);
  if (bytes > fr / 3) { l.pk_fail = want_w; return; }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); l.pk_fail = want_w; return; }
  s.pk_base = p;
  s.wpk = (double*)p;
  s.bpt = s.wpk + want_w;
  s.wpk_cap = want_w;
  s.bpt_cap = want_b;
}

int ensure_scratch(molgw_ctx c, Lane& l, int nb, int na, long long nov) {
  Scratch& s = l.scr;
  const size_t want_w = std::max<size_t>((size_t)nb * nov,
                                         std::min<size_t>((size_t)nb * nb * nov, (size_t)48 << 20));
  if (!use_tc(c) && !use_mp2(c)) ensure_packed(c, l, nb, na, nov);
  if (nb <= s.nb_cap && na <= s.na_cap && want_w <= s.wblk_cap) return MOLGW_OK;
  if (l.ex.capturing) return MOLGW_E_STATE;
  cudaStreamSynchronize(l.st);
  ++c->gen;
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

// Arena of the orbital-size split operands (tensor-core path).
int ensure_tco(molgw_ctx c, Lane& l, int nb, int na, long long nov) {
  if (!use_tc(c)) return MOLGW_OK;
  const int prec = tc_prec(c);
  const bool mp2 = use_mp2(c);
  const size_t want = use_fx(c) ? (std::max(fx_sigma_bytes(nb, na, nov, fx_mblock(nb, na, nov, mp2), mp2),
                                            use_tc_ab(c) ? fx_ab_bytes(nb, na, nov) : (size_t)0) + 7) / 8
                                : tc_orb_doubles(prec, nb, na, nov, tc_mblock(prec, nb, nov));
  if (want <= l.tco_cap) return MOLGW_OK;
  if (l.ex.capturing) return MOLGW_E_STATE;
  cudaStreamSynchronize(l.st);
  ++c->gen;
  if (l.tco_base) cudaFree(l.tco_base);
  l.tco_base = nullptr;
  l.tco_cap = 0;
  if (cudaMalloc(&l.tco_base, want * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    l.tco_base = nullptr;
    return MOLGW_E_NOMEM;
  }
  l.tco_cap = want;
  return MOLGW_OK;
}

// Every buffer one pass of molecule m needs on lane l.
int lane_fit(molgw_ctx c, Lane& l, const MolBuf& m) {
  const bool full = (c->opts.flags & MOLGW_FLAG_FULL_XPY) != 0;
  int r = ensure_scratch(c, l, m.nb, m.na, m.nov);
  if (!r && use_mp2(c)) r = ensure_eig(c, l, m.nb, m.nb);   // qs_update only
  else if (!r) r = ensure_eig(c, l, (int)std::max<long long>(m.nov, m.nb),
                              std::max<int>(std::max(m.na, m.nb), full ? (int)m.nov : 0));
  if (!r) r = ensure_eigfx(c, l);
  if (!r) r = ensure_tco(c, l, m.nb, m.na, m.nov);
  return r;
}

// An NVTX range over one stage of a pass (shown by Nsight tools; free without one).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// Open shell (float64, or BF16X10 with the contractions on the fixed-point engine):
// both spin channels through (a), J, Sigma_x and h; one RPA over the transitions of
// both spins (up first); (d)+(e) and (f) per channel, the spin-down channel reading
// R and Omega of the spin-up MolBuf.
int run_pass_open(molgw_ctx c, Lane& l, int mol, char upto) {
  MolBuf& m = c->mols[mol];
  MolBuf& d = *m.dn;
  if (upto == 'g') return MOLGW_E_STATE;   // G0W0 is closed-shell only
  int r = lane_fit(c, l, m);
  if (r) return r;
  Exec& ex = l.ex;
  const bool fx = use_fx(c), fx_ab = fx && use_tc_ab(c);
  if (fx) fx_bufs_carve(l.fxo, m.nb, m.na, m.nov, fx_mblock(m.nb, m.na, m.nov), l.tco_base);
  if (!m.b_valid) {
    Range rg("(a) ri_mo_transform, both spins");
    if (fx_ab) {
      r = stage_ri_mo_transform_fx(ex, m, c->tcb[mol].Lfx, l.tco_base);
      if (!r) r = stage_ri_mo_transform_fx(ex, d, c->tcb[mol].Lfx, l.tco_base);
      if (r) return r;
    } else {
      stage_ri_mo_transform(ex, m);
      stage_ri_mo_transform(ex, d);
    }
    m.b_valid = m.have_b = true;
  }
  if (!m.h_ready) {
    Range rg("J, Sigma_x, h_MO, both spins");
    stage_j_sigx(ex, m, l.scr, &d);
    stage_j_sigx(ex, d, l.scr, &m);
    derive_h_from_hf(ex, m);
    derive_h_from_hf(ex, d);
    m.jx_valid = m.have_jx = true;
    m.h_ready = true;
  }
  if (upto == 'b' || !m.rpa_valid) {
    {
      Range rg("(b) rpa_build");
      if (fx_ab) {
        r = stage_rpa_build_fx(ex, m, l.tco_base);
        if (r) return r;
      } else {
        stage_rpa_build(ex, m);
      }
    }
    if (upto == 'b') {
      m.rpa_valid = false;
      return launch_status();
    }
    Range rg("(c) rpa_eigensolve");
    stage_rpa_eigensolve(ex, m, l.eig, l.scr, false);
    m.rpa_valid = m.have_rpa = true;
  }
  if (upto >= 'e' && !m.sigma_valid) {
    Range rg("(d)+(e) gw_residues, sigma_assembly, both spins");
    if (!m.jx_valid) {
      stage_j_sigx(ex, m, l.scr, &d);
      stage_j_sigx(ex, d, l.scr, &m);
      m.jx_valid = m.have_jx = true;
    }
    if (fx) {
      r = stage_sigma_fx(ex, m, l.fxo, l.scr, c->opts.eta);
      if (!r) r = stage_sigma_fx(ex, d, l.fxo, l.scr, c->opts.eta);
      if (r) return r;
    } else {
      stage_sigma(ex, m, l.scr, c->opts.eta);
      stage_sigma(ex, d, l.scr, c->opts.eta);
    }
    m.sigma_valid = m.have_sigma = true;
  }
  if (upto == 'f') {
    Range rg("(f) qs_update, both spins");
    stage_qs_update(ex, m, l.eig, l.scr);
    stage_qs_update(ex, d, l.eig, l.scr);
    m.b_valid = m.jx_valid = m.rpa_valid = m.sigma_valid = false;
  }
  return launch_status();
}

// Run the pass of one molecule on lane l up to a stage: 'b' (M), 'c' (rpa),
// 'e' (sigma), 'f' (qs step).
int run_pass(molgw_ctx c, Lane& l, int mol, char upto) {
  MolBuf& m = c->mols[mol];
  if (!m.have_ri || !m.have_orb) return MOLGW_E_STATE;
  if (m.dn) return run_pass_open(c, l, mol, upto);
  const bool mp2 = use_mp2(c);
  if (mp2 && (upto < 'e' || upto == 'g')) return MOLGW_E_STATE;   // qsMP2 has no RPA stages
  const bool full = (c->opts.flags & MOLGW_FLAG_FULL_XPY) != 0;
  int r = lane_fit(c, l, m);
  if (r) return r;
  Exec& ex = l.ex;
  const bool tc = use_tc(c);
  const bool tc_ab = use_tc_ab(c);
  TcBufs& tb = l.tco;
  if (use_fx(c)) {
    fx_bufs_carve(l.fxo, m.nb, m.na, m.nov, fx_mblock(m.nb, m.na, m.nov, mp2), l.tco_base, mp2, m.no);
  } else if (tc) {
    const int prec = tc_prec(c);
    tc_bufs_carve(tb, prec, m.nb, m.na, m.nov, tc_mblock(prec, m.nb, m.nov), (double*)l.tco_base);
    tb.L = c->tcb[mol].L;
  }
  if (!m.b_valid) {
    Range rg("(a) ri_mo_transform");
    if (tc_ab && use_fx(c)) {
      r = stage_ri_mo_transform_fx(ex, m, c->tcb[mol].Lfx, l.tco_base);
      if (r) return r;
    } else if (tc_ab) {
      r = stage_ri_mo_transform_tc(ex, m, tb);
      if (r) return r;
    } else {
      stage_ri_mo_transform(ex, m);
    }
    m.b_valid = m.have_b = true;
  }
  if (!m.h_ready) {
    Range rg("J, Sigma_x, h_MO");
    stage_j_sigx(ex, m, l.scr);
    derive_h_from_hf(ex, m);
    m.jx_valid = m.have_jx = true;
    m.h_ready = true;
  }
  if (upto == 'b') {
    Range rg("(b) rpa_build");
    if (tc_ab && use_fx(c)) {
      r = stage_rpa_build_fx(ex, m, l.tco_base);
      if (r) return r;
    } else if (tc_ab) {
      r = stage_rpa_build_tc(ex, m, tb);
      if (r) return r;
    } else {
      stage_rpa_build(ex, m);
    }
    m.rpa_valid = false;
    return launch_status();
  }
  if (!m.rpa_valid && !mp2) {
    {
      Range rg("(b) rpa_build");
      if (tc_ab && use_fx(c)) {
        r = stage_rpa_build_fx(ex, m, l.tco_base);
        if (r) return r;
      } else if (tc_ab) {
        r = stage_rpa_build_tc(ex, m, tb);
        if (r) return r;
      } else {
        stage_rpa_build(ex, m);
      }
    }
    Range rg("(c) rpa_eigensolve");
    stage_rpa_eigensolve(ex, m, l.eig, l.scr, full);
    m.rpa_valid = m.have_rpa = true;
  }
  if (upto == 'g') {
    // one-shot G0W0 from the current orbitals; they stay current
    Range rg("G0W0");
    if (!m.jx_valid) {
      stage_j_sigx(ex, m, l.scr);
      m.jx_valid = m.have_jx = true;
    }
    r = stage_g0w0(ex, m, l.scr, c->opts.eta, std::min(c->g0w0_p0, m.nb), std::min(c->g0w0_p1, m.nb));
    if (r) return r;
    m.have_g0w0 = true;
    return launch_status();
  }
  if (upto >= 'e' && !m.sigma_valid) {
    Range rg(mp2 ? "(d)+(e) qsMP2 self-energy" : "(d)+(e) gw_residues, sigma_assembly");
    if (!m.jx_valid) {
      stage_j_sigx(ex, m, l.scr);
      m.jx_valid = m.have_jx = true;
    }
    if (mp2 && use_fx(c)) {
      r = stage_sigma_mp2_fx(ex, m, l.fxo, l.scr, c->opts.eta);
      if (r) return r;
    } else if (mp2) {
      stage_sigma_mp2(ex, m, l.scr, c->opts.eta);
    } else if (use_fx(c)) {
      r = stage_sigma_fx(ex, m, l.fxo, l.scr, c->opts.eta);
      if (r) return r;
    } else if (tc) {
      r = stage_sigma_tc(ex, m, tb, l.scr, c->opts.eta);
      if (r) return r;
    } else {
      stage_sigma(ex, m, l.scr, c->opts.eta);
    }
    m.sigma_valid = m.have_sigma = true;
  }
  if (upto == 'f') {
    Range rg("(f) qs_update");
    stage_qs_update(ex, m, l.eig, l.scr);
    m.b_valid = m.jx_valid = m.rpa_valid = m.sigma_valid = false;
  }
  return launch_status();
}

bool ready(const MolBuf& m) { return m.have_ri && m.have_orb; }

// The state a qs_step leaves behind: the next qs_step issues exactly the same
// launches, so a graph captured from one replays the next.
bool steady(const MolBuf& m) {
  return ready(m) && m.h_ready && !m.b_valid && !m.jx_valid && !m.rpa_valid && !m.sigma_valid;
}

// Relative cost of one pass: the n_ov^3 eigensolve and the residue contraction (one per
// spin channel); for qsMP2 the direct and exchange factors and the Sigma contraction.
double pass_cost_of(long long nb, long long na, long long nov, bool open, bool mp2) {
  const double n = (double)nov, b = (double)nb, a = (double)na;
  if (mp2) return 2.0 * 2.0 * b * b * n * a + 2.0 * b * b * b * n;
  return n * n * n + (open ? 2.0 : 1.0) * 2.0 * b * b * n * a;
}

double pass_cost(const MolBuf& m, bool mp2) { return pass_cost_of(m.nb, m.na, m.nov, m.dn != nullptr, mp2); }

// Longest-processing-time-first: items in order of decreasing cost (equal costs by
// index), each to the lane with the least load so far (equal loads: the lowest lane).
// Returns the items of each of the max(1, min(lanes, items)) lanes in issue order.
std::vector<std::vector<int>> lpt_assign(const std::vector<double>& cost, int lanes) {
  const int n = (int)cost.size();
  const int nl = std::max(1, std::min(lanes, n));
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<std::vector<int>> out(nl);
  std::vector<double> load(nl, 0.0);
  for (int k : order) {
    int best = 0;
    for (int j = 1; j < nl; ++j)
      if (load[j] < load[best]) best = j;
    out[best].push_back(k);
    load[best] += cost[k];
  }
  return out;
}

struct Plan {
  std::vector<std::vector<int>> lane_mols;   // molecules of each lane, in issue order
};

int lanes_wanted(molgw_ctx c) {
  if (c->opts.lanes > 0) return std::min(c->opts.lanes, kMaxLanes);
  return c->tuned_lanes > 0 ? c->tuned_lanes : kDefaultLanes;
}

// The molecules spread over at most `lanes` (0: lanes_wanted) lanes by lpt_assign.
Plan plan_batch(molgw_ctx c, const std::vector<int>& mols, int lanes = 0) {
  const int want = std::min(lanes > 0 ? lanes : lanes_wanted(c), kMaxLanes);
  std::vector<double> cost;
  for (int k : mols) cost.push_back(pass_cost(c->mols[k], use_mp2(c)));
  Plan p;
  for (const auto& items : lpt_assign(cost, want)) {
    p.lane_mols.emplace_back();
    for (int i : items) p.lane_mols.back().push_back(mols[i]);
  }
  return p;
}

// Create the lanes of a plan and size their buffers for their molecules (no
// allocation happens while the passes are issued).
int plan_fit(molgw_ctx c, const Plan& p) {
  for (int k = 0; k < (int)p.lane_mols.size(); ++k) {
    Lane* l = nullptr;
    int r = lane_get(c, k, &l);
    if (r) return r;
    for (int mol : p.lane_mols[k]) {
      r = lane_fit(c, c->lanes[k], c->mols[mol]);
      if (r) return r;
    }
  }
  return MOLGW_OK;
}

// Issue the passes of a plan: the lanes fork from the context stream, each runs
// its molecules in order (issued round robin across lanes), and the context
// stream waits for all of them.  With several lanes each persistent panel
// launch is limited to an equal share of the co-resident CTAs.
int issue_plan(molgw_ctx c, const Plan& p, char upto) {
  const int nl = (int)p.lane_mols.size();
  const int share = nl > 1 ? tridiag_coop_capacity() / nl : 0;
  for (int k = 0; k < nl; ++k) c->lanes[k].ex.coop_cap = share;
  if (nl > 1) {
    cudaEventRecord(c->fork, c->st);
    for (int k = 1; k < nl; ++k) cudaStreamWaitEvent(c->lanes[k].st, c->fork, 0);
  }
  int r = MOLGW_OK;
  size_t depth = 0;
  for (const auto& v : p.lane_mols) depth = std::max(depth, v.size());
  for (size_t i = 0; i < depth && !r; ++i)
    for (int k = 0; k < nl && !r; ++k)
      if (i < p.lane_mols[k].size()) r = run_pass(c, c->lanes[k], p.lane_mols[k][i], upto);
  if (nl > 1) {
    // join even after an error, so that no lane is left outside the context stream's order
    for (int k = 1; k < nl; ++k) {
      cudaEventRecord(c->lanes[k].done, c->lanes[k].st);
      cudaStreamWaitEvent(c->st, c->lanes[k].done, 0);
    }
  }
  for (int k = 0; k < nl; ++k) c->lanes[k].ex.coop_cap = 0;
  if (!r) r = launch_status();
  return r;
}

void graph_drop(molgw_ctx c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->graph_mol = -2;
  c->graph_gen = 0;
  c->graph_set.clear();
}

std::vector<char> mol_set(molgw_ctx c, const std::vector<int>& mols) {
  std::vector<char> v(c->mols.size(), 0);
  for (int k : mols) v[k] = 1;
  return v;
}

struct Flags {
  bool h_ready, b_valid, jx_valid, rpa_valid, sigma_valid, have_b, have_rpa, have_jx, have_sigma;
};
Flags get_flags(const MolBuf& m) {
  return {m.h_ready, m.b_valid, m.jx_valid, m.rpa_valid, m.sigma_valid, m.have_b, m.have_rpa, m.have_jx, m.have_sigma};
}
void put_flags(MolBuf& m, const Flags& f) {
  m.h_ready = f.h_ready; m.b_valid = f.b_valid; m.jx_valid = f.jx_valid; m.rpa_valid = f.rpa_valid;
  m.sigma_valid = f.sigma_valid; m.have_b = f.have_b; m.have_rpa = f.have_rpa; m.have_jx = f.have_jx;
  m.have_sigma = f.have_sigma;
}

// Capture the qs_step passes of a plan into c->gexec.  Returns false (and turns
// graphs off for the context) when the capture or the instantiation fails; the
// caller then issues the passes directly.
bool graph_capture(molgw_ctx c, int mol, const std::vector<int>& mols, const Plan& p) {
  graph_drop(c);
  std::vector<Flags> saved;
  for (int k : mols) saved.push_back(get_flags(c->mols[k]));
  int64_t before[MOLGW_K_COUNT];
  for (int k = 0; k < MOLGW_K_COUNT; ++k) before[k] = c->timer.launches[k];
  const int64_t total_before = c->timer.total_launches;
  bool ok = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  cudaGraph_t g = nullptr;
  if (ok) {
    for (auto& l : c->lanes) l.ex.capturing = true;
    const int r = issue_plan(c, p, 'f');
    for (auto& l : c->lanes) l.ex.capturing = false;
    const cudaError_t e = cudaStreamEndCapture(c->st, &g);
    ok = (r == MOLGW_OK) && e == cudaSuccess && g != nullptr;
  }
  for (size_t i = 0; i < mols.size(); ++i) put_flags(c->mols[mols[i]], saved[i]);
  for (int k = 0; k < MOLGW_K_COUNT; ++k) {
    c->graph_launches[k] = c->timer.launches[k] - before[k];
    c->timer.launches[k] = before[k];
  }
  c->timer.total_launches = total_before;
  if (ok) ok = cudaGraphInstantiate(&c->gexec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    c->gexec = nullptr;
    c->graph_off = true;
    return false;
  }
  c->graph_mol = mol;
  c->graph_gen = c->gen;
  c->graph_set = mol_set(c, mols);
  c->graph_lanes = (int)p.lane_mols.size();
  return true;
}

// Stages up to `upto` for molecule `mol`, or for every ready molecule (mol = -1)
// spread over concurrent lanes.  With MOLGW_FLAG_GRAPH a qs_step from the steady
// state is captured once and replayed while the buffers and the set of molecules
// stay the same.
int run_mols(molgw_ctx c, int mol, char upto) {
  std::vector<int> mols;
  if (mol == -1) {
    for (int k = 0; k < (int)c->mols.size(); ++k)
      if (ready(c->mols[k])) mols.push_back(k);
    if (mols.empty()) return MOLGW_E_STATE;
  } else {
    if (!ready(c->mols[mol])) return MOLGW_E_STATE;
    mols.push_back(mol);
  }
  Plan p = plan_batch(c, mols);
  int r = plan_fit(c, p);
  if (r) return r;
  bool graph = upto == 'f' && (c->opts.flags & MOLGW_FLAG_GRAPH) && !c->graph_off;
  for (int k : mols) graph = graph && steady(c->mols[k]);
  if (!graph) return issue_plan(c, p, upto);
  const bool match = c->gexec && c->graph_mol == mol && c->graph_gen == c->gen && c->graph_set == mol_set(c, mols) &&
                     c->graph_lanes == (int)p.lane_mols.size();
  if (!match && !graph_capture(c, mol, mols, p)) return issue_plan(c, p, upto);
  if (cudaGraphLaunch(c->gexec, c->st) != cudaSuccess) return cuda_status(cudaGetLastError());
  ++c->graph_replays;
  for (int k : mols) {
    MolBuf& m = c->mols[k];
    m.have_b = m.have_rpa = m.have_jx = m.have_sigma = true;
    m.b_valid = m.jx_valid = m.rpa_valid = m.sigma_valid = false;
  }
  for (int k = 0; k < MOLGW_K_COUNT; ++k) {
    c->timer.launches[k] += c->graph_launches[k];
    c->timer.total_launches += c->graph_launches[k];
  }
  return MOLGW_OK;
}

}  // namespace

extern "C" {

int molgw_b200_create(const molgw_opts* o, molgw_ctx* out) {
  if (!out) return MOLGW_E_ARG;
  *out = nullptr;
  if (!o || o->struct_size != (int32_t)sizeof(molgw_opts)) return MOLGW_E_ARG;
  if (o->precision < MOLGW_PREC_FP64 || o->precision > MOLGW_PREC_BF16X10) return MOLGW_E_ARG;
  if (o->max_mols < 1 || !(o->eta > 0.0) || o->lanes < 0) return MOLGW_E_ARG;
  if ((o->flags & MOLGW_FLAG_QSMP2) && o->precision != MOLGW_PREC_FP64 && o->precision != MOLGW_PREC_BF16X10)
    return MOLGW_E_ARG;
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
  Lane* l0 = nullptr;
  if (cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess || lane_get(c, 0, &l0) != MOLGW_OK) {
    cudaGetLastError();
    molgw_b200_destroy(c);
    return MOLGW_E_CUDA;
  }
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
  m.have_b = m.have_rpa = m.have_jx = m.have_sigma = m.have_g0w0 = false;
  m.h_ready = false;
  if (m.dn) {
    cudaStreamSynchronize(c->st);
    ++c->gen;
    drop_open(m);
    free_all(m.orb_allocs);
    m.eps = nullptr;
    m.alloc_no = 0;
  }
  if (m.ri_allocs.empty() || m.nb != n_basis || m.na != n_aux) {
    cudaStreamSynchronize(c->st);
    ++c->gen;
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
    if (use_tc_ab(c) && use_fx(c)) {
      const long long rows = (long long)n_aux * n_basis, ld = fx_pad(n_basis);
      double* base = dalloc(tb.ri_allocs, (fx_mat_bytes(rows, ld) + 7) / 8, &err);
      if (!err) tb.Lfx = fx_mat_carve(base, rows, ld);
    } else if (use_tc_ab(c)) {
      double* base = dalloc(tb.ri_allocs, tc_ri_doubles(tc_prec(c), n_basis, n_aux), &err);
      if (!err) tc_ri_carve(tb, tc_prec(c), n_basis, n_aux, base);
    }
    if (err) { free_all(m.ri_allocs); free_all(tb.ri_allocs); m.nb = m.na = 0; return err; }
  }
  int r = copy_in(c, m.L, L, nl);
  if (r) return r;
  Exec& ex = c->lanes[0].ex;
  check_finite(ex, m.L, (long long)nl);
  if (use_tc_ab(c) && use_fx(c))
    fx_split(ex, m.L, (long long)n_aux * n_basis, n_basis, n_basis, 1, nullptr, c->tcb[mol].Lfx);
  else if (use_tc_ab(c))
    tc_split_ri(ex, m, c->tcb[mol]);
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
  if (m.orb_allocs.empty() || m.alloc_no != n_occ || m.dn) {
    cudaStreamSynchronize(c->st);
    ++c->gen;
    drop_open(m);
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
    m.g0w0 = dalloc(m.orb_allocs, 3 * (size_t)nb, &err);
    m.D = dalloc(m.orb_allocs, nov, &err);
    m.Om = dalloc(m.orb_allocs, nov, &err);
    m.R = dalloc(m.orb_allocs, (size_t)nov * na, &err);     // qsMP2: B_ia
    if (use_mp2(c)) {
      m.Xv = m.M = m.ZT = m.XpY = nullptr;                   // no RPA
    } else {
      m.Xv = dalloc(m.orb_allocs, (size_t)nov * na, &err);
      m.M = dalloc(m.orb_allocs, (size_t)nov * nov, &err);
      m.ZT = dalloc(m.orb_allocs, (size_t)nov * nov, &err);
      m.XpY = full ? dalloc(m.orb_allocs, (size_t)nov * nov, &err) : nullptr;
    }
    if (err) { free_all(m.orb_allocs); m.eps = nullptr; m.alloc_no = 0; return err; }
    m.alloc_no = n_occ;
  }
  m.no = n_occ;
  m.nov = nov;
  int r = copy_in(c, m.eps, eps, nb);
  if (!r) r = copy_in(c, m.C, C, (size_t)nb * nb);
  if (r) return r;
  Exec& ex = c->lanes[0].ex;
  check_finite(ex, m.eps, nb);
  check_finite(ex, m.C, (long long)nb * nb);
  // all-ones bytes are a NaN: G0W0 entries that no window has computed for these orbitals
  cudaMemsetAsync(m.g0w0, 0xFF, 3 * (size_t)nb * sizeof(double), c->st);
  m.have_orb = true;
  m.b_valid = m.jx_valid = m.rpa_valid = m.sigma_valid = false;
  m.have_b = m.have_rpa = m.have_jx = m.have_sigma = m.have_g0w0 = false;
  m.h_ready = false;
  if (h_core) {
    r = ensure_scratch(c, c->lanes[0], nb, na, nov);
    if (r) return r;
    // stage h_AO in the T1 buffer (n_aux*nb*nb >= nb*nb), then h_MO = C^T h C
    r = copy_in(c, m.T1, h_core, (size_t)nb * nb);
    if (r) return r;
    h_ao_to_mo(ex, m, m.T1, c->lanes[0].scr);
    m.h_ready = true;
  }
  return launch_status();
}

int molgw_b200_set_orbitals_open(molgw_ctx c, int mol, int n_occ_up, int n_occ_dn, const double* eps_up,
                                 const double* eps_dn, const double* C_up, const double* C_dn,
                                 const double* h_core) {
  if (!mol_ok(c, mol) || !eps_up || !eps_dn || !C_up || !C_dn) return MOLGW_E_ARG;
  if ((c->opts.precision != MOLGW_PREC_FP64 && c->opts.precision != MOLGW_PREC_BF16X10) ||
      (c->opts.flags & (MOLGW_FLAG_QSMP2 | MOLGW_FLAG_FULL_XPY)))
    return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  MolBuf& m = c->mols[mol];
  if (!m.have_ri) return MOLGW_E_STATE;
  const int nb = m.nb, na = m.na;
  if (n_occ_up < 0 || n_occ_dn < 0 || n_occ_up >= nb || n_occ_dn >= nb || n_occ_up + n_occ_dn < 1)
    return MOLGW_E_ARG;
  const long long nov_up = (long long)n_occ_up * (nb - n_occ_up);
  const long long nov = nov_up + (long long)n_occ_dn * (nb - n_occ_dn);
  const int key = -(1 + n_occ_up * 65536 + n_occ_dn);    // allocation key of this occupation pair
  const size_t nn = (size_t)nb * nb;
  if (m.orb_allocs.empty() || m.alloc_no != key || !m.dn) {
    cudaStreamSynchronize(c->st);
    ++c->gen;
    drop_open(m);
    free_all(m.orb_allocs);
    m.have_orb = false;
    int err = 0;
    m.eps = dalloc(m.orb_allocs, nb, &err);
    m.C = dalloc(m.orb_allocs, nn, &err);
    m.hmo = dalloc(m.orb_allocs, nn, &err);
    m.J = dalloc(m.orb_allocs, nn, &err);
    m.sigx = dalloc(m.orb_allocs, nn, &err);
    m.sigc = dalloc(m.orb_allocs, nn, &err);
    m.g0w0 = nullptr;
    m.D = dalloc(m.orb_allocs, nov, &err);
    m.Om = dalloc(m.orb_allocs, nov, &err);
    m.R = dalloc(m.orb_allocs, (size_t)nov * na, &err);
    m.Xv = dalloc(m.orb_allocs, (size_t)nov * na, &err);
    m.M = dalloc(m.orb_allocs, (size_t)nov * nov, &err);
    m.ZT = dalloc(m.orb_allocs, (size_t)nov * nov, &err);
    m.XpY = nullptr;
    std::unique_ptr<MolBuf> d(new (std::nothrow) MolBuf());
    if (!d) err = MOLGW_E_NOMEM;
    if (!err) {
      d->B = dalloc(d->ri_allocs, (size_t)na * nn, &err);
      d->T1 = dalloc(d->ri_allocs, (size_t)na * nn, &err);
      d->eps = dalloc(d->orb_allocs, nb, &err);
      d->C = dalloc(d->orb_allocs, nn, &err);
      d->hmo = dalloc(d->orb_allocs, nn, &err);
      d->J = dalloc(d->orb_allocs, nn, &err);
      d->sigx = dalloc(d->orb_allocs, nn, &err);
      d->sigc = dalloc(d->orb_allocs, nn, &err);
    }
    if (err) {
      if (d) { free_all(d->ri_allocs); free_all(d->orb_allocs); }
      free_all(m.orb_allocs);
      m.eps = nullptr;
      m.alloc_no = 0;
      return err;
    }
    m.dn = std::move(d);
    m.alloc_no = key;
  }
  MolBuf& d = *m.dn;
  m.no = n_occ_up;
  m.nov = nov;
  m.nov_up = nov_up;
  // the spin-down channel: its own orbitals and B, the RI factors and the RPA of m
  d.nb = nb; d.na = na; d.no = n_occ_dn; d.nov = nov;
  d.L = m.L; d.R = m.R; d.Om = m.Om; d.D = m.D;
  d.have_ri = d.have_orb = true;
  int r = copy_in(c, m.eps, eps_up, nb);
  if (!r) r = copy_in(c, m.C, C_up, nn);
  if (!r) r = copy_in(c, d.eps, eps_dn, nb);
  if (!r) r = copy_in(c, d.C, C_dn, nn);
  if (r) return r;
  Exec& ex = c->lanes[0].ex;
  check_finite(ex, m.eps, nb);
  check_finite(ex, m.C, (long long)nn);
  check_finite(ex, d.eps, nb);
  check_finite(ex, d.C, (long long)nn);
  m.have_orb = true;
  m.b_valid = m.jx_valid = m.rpa_valid = m.sigma_valid = false;
  m.have_b = m.have_rpa = m.have_jx = m.have_sigma = m.have_g0w0 = false;
  m.h_ready = false;
  if (h_core) {
    r = ensure_scratch(c, c->lanes[0], nb, na, nov);
    if (r) return r;
    r = copy_in(c, m.T1, h_core, nn);
    if (r) return r;
    h_ao_to_mo(ex, m, m.T1, c->lanes[0].scr);
    h_ao_to_mo(ex, d, m.T1, c->lanes[0].scr);
    m.h_ready = true;
  }
  return launch_status();
}

int molgw_b200_rpa(molgw_ctx c, int mol, double* omega, double* xpy) {
  if (!c) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  if (mol == -1) {
    if (omega || xpy) return MOLGW_E_ARG;
    return run_mols(c, -1, 'c');
  }
  if (!mol_ok(c, mol)) return MOLGW_E_ARG;
  if (xpy && !(c->opts.flags & MOLGW_FLAG_FULL_XPY)) return MOLGW_E_ARG;
  MolBuf& m = c->mols[mol];
  if (!ready(m)) return MOLGW_E_STATE;
  int r = run_mols(c, mol, 'c');
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
    return run_mols(c, -1, 'e');
  }
  if (!mol_ok(c, mol)) return MOLGW_E_ARG;
  MolBuf& m = c->mols[mol];
  if (!ready(m)) return MOLGW_E_STATE;
  int r = run_mols(c, mol, 'e');
  if (r) return r;
  bool sync = false;
  const size_t nn = (size_t)m.nb * m.nb;
  if (sigma_x) r = copy_out(c, sigma_x, m.sigx, nn, &sync);
  if (!r && sigma_c) r = copy_out(c, sigma_c, m.sigc, nn, &sync);
  if (m.dn) {   // open shell: the spin-down blocks follow
    if (!r && sigma_x) r = copy_out(c, sigma_x + nn, m.dn->sigx, nn, &sync);
    if (!r && sigma_c) r = copy_out(c, sigma_c + nn, m.dn->sigc, nn, &sync);
  }
  if (r) return r;
  return sync ? read_status(c) : MOLGW_OK;
}

int molgw_b200_g0w0_window(molgw_ctx c, int mol, int p_begin, int p_end, double* eps_qp, double* z,
                           double* sigma_c_diag) {
  if (!c || p_begin < 0 || p_end <= p_begin) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  c->g0w0_p0 = p_begin;
  c->g0w0_p1 = p_end;
  if (mol == -1) {
    if (eps_qp || z || sigma_c_diag) return MOLGW_E_ARG;
    return run_mols(c, -1, 'g');
  }
  if (!mol_ok(c, mol)) return MOLGW_E_ARG;
  MolBuf& m = c->mols[mol];
  if (!ready(m)) return MOLGW_E_STATE;
  if (p_end > m.nb) return MOLGW_E_ARG;
  int r = run_mols(c, mol, 'g');
  if (r) return r;
  bool sync = false;
  const int np = p_end - p_begin;
  if (eps_qp) r = copy_out(c, eps_qp, m.g0w0 + p_begin, np, &sync);
  if (!r && z) r = copy_out(c, z, m.g0w0 + m.nb + p_begin, np, &sync);
  if (!r && sigma_c_diag) r = copy_out(c, sigma_c_diag, m.g0w0 + 2 * m.nb + p_begin, np, &sync);
  if (r) return r;
  return sync ? read_status(c) : MOLGW_OK;
}

int molgw_b200_g0w0(molgw_ctx c, int mol, double* eps_qp, double* z, double* sigma_c_diag) {
  if (!c) return MOLGW_E_ARG;
  const int nb = (mol >= 0 && mol_ok(c, mol)) ? c->mols[mol].nb : (1 << 30);
  return molgw_b200_g0w0_window(c, mol, 0, nb, eps_qp, z, sigma_c_diag);
}

int molgw_b200_qs_step(molgw_ctx c, int mol, double* eps_out, double* C_out) {
  if (!c) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  if (mol == -1) {
    if (eps_out || C_out) return MOLGW_E_ARG;
    return run_mols(c, -1, 'f');
  }
  if (!mol_ok(c, mol)) return MOLGW_E_ARG;
  MolBuf& m = c->mols[mol];
  if (!ready(m)) return MOLGW_E_STATE;
  int r = run_mols(c, mol, 'f');
  if (r) return r;
  bool sync = false;
  if (eps_out) r = copy_out(c, eps_out, m.eps, m.nb, &sync);
  if (!r && C_out) r = copy_out(c, C_out, m.C, (size_t)m.nb * m.nb, &sync);
  if (m.dn) {   // open shell: the spin-down energies and orbitals follow
    if (!r && eps_out) r = copy_out(c, eps_out + m.nb, m.dn->eps, m.nb, &sync);
    if (!r && C_out) r = copy_out(c, C_out + (size_t)m.nb * m.nb, m.dn->C, (size_t)m.nb * m.nb, &sync);
  }
  if (r) return r;
  return sync ? read_status(c) : MOLGW_OK;
}

int molgw_b200_sync(molgw_ctx c) {
  if (!c) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  return read_status(c);
}

int molgw_b200_inject_fault(molgw_ctx c, int code) {
  if (!c || (code != MOLGW_E_TIMEOUT && code != MOLGW_E_NOCONV && code != MOLGW_E_NUMERIC)) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  k_inject_status<<<1, 1, 0, c->st>>>(c->d_status, code);
  return launch_status();
}

int molgw_b200_set_wait_limits(molgw_ctx c, long long grid_spins, int bisect_rounds) {
  if (!c) return MOLGW_E_ARG;
  c->grid_spins = grid_spins < 0 ? kGridSpinLimit : grid_spins;
  c->bisect_rounds = bisect_rounds < 0 ? kBisectRounds : std::min(bisect_rounds, kBisectRounds);
  for (Lane& l : c->lanes) {
    l.ex.grid_spins = c->grid_spins;
    l.ex.bisect_rounds = c->bisect_rounds;
  }
  ++c->gen;   // a captured graph holds the old bounds in its launch parameters
  return MOLGW_OK;
}

int molgw_b200_set_panel_matvec(molgw_ctx c, int kind) {
  if (!c || kind < MOLGW_MATVEC_AUTO || kind > MOLGW_MATVEC_INT) return MOLGW_E_ARG;
  c->panel_matvec = kind;
  for (Lane& l : c->lanes) l.ex.panel_matvec = kind;
  ++c->gen;   // a captured graph holds the old choice in its launches
  return MOLGW_OK;
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
    case MOLGW_ITEM_EPS_QP: src = m.g0w0; n = m.nb; avail = m.have_g0w0; break;
    case MOLGW_ITEM_Z: src = m.g0w0 + m.nb; n = m.nb; avail = m.have_g0w0; break;
    case MOLGW_ITEM_SIGMA_C_DIAG: src = m.g0w0 + 2 * m.nb; n = m.nb; avail = m.have_g0w0; break;
    default: return MOLGW_E_ARG;
  }
  if (!avail) return MOLGW_E_STATE;
  // open shell: the per-orbital items are the spin-up block followed by the spin-down one
  const double* src_dn = nullptr;
  if (m.dn) {
    const MolBuf& d = *m.dn;
    switch (item) {
      case MOLGW_ITEM_B: src_dn = d.B; break;
      case MOLGW_ITEM_SIGMA_X: src_dn = d.sigx; break;
      case MOLGW_ITEM_SIGMA_C: src_dn = d.sigc; break;
      case MOLGW_ITEM_J: src_dn = d.J; break;
      case MOLGW_ITEM_H_MO: src_dn = d.hmo; break;
      case MOLGW_ITEM_EPS: src_dn = d.eps; break;
      case MOLGW_ITEM_C: src_dn = d.C; break;
      case MOLGW_ITEM_OMEGA: case MOLGW_ITEM_R: break;
      default: return MOLGW_E_STATE;             // G0W0 items: closed shell only
    }
  }
  if (count != (src_dn ? 2 * n : n)) return MOLGW_E_ARG;
  bool sync = false;
  int r = copy_out(c, out, src, n, &sync);
  if (!r && src_dn) r = copy_out(c, out + n, src_dn, n, &sync);
  if (r) return r;
  return sync ? read_status(c) : MOLGW_OK;
}

int molgw_b200_rpa_matrix(molgw_ctx c, int mol, double* M) {
  if (!mol_ok(c, mol) || !M) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  MolBuf& m = c->mols[mol];
  if (!ready(m)) return MOLGW_E_STATE;
  int r = run_mols(c, mol, 'b');
  if (r) return r;
  // the build keeps the lower 64x64 tiles and full diagonal tiles: mirror them
  fill_upper(c->lanes[0].ex, m.M, m.nov);
  bool sync = false;
  r = copy_out(c, M, m.M, (size_t)m.nov * m.nov, &sync);
  if (r) return r;
  return sync ? read_status(c) : MOLGW_OK;
}

int molgw_b200_eigh(molgw_ctx c, int n, const double* A, double* w, double* Z) {
  if (!c || n < 1 || !A || !w) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  Lane& l = c->lanes[0];
  int r = ensure_eig(c, l, n, n);
  if (!r) r = ensure_eigfx(c, l);
  if (r) return r;
  std::vector<void*> tmp;
  int err = 0;
  double* dA = dalloc(tmp, (size_t)n * n, &err);
  double* dZ = Z ? dalloc(tmp, (size_t)n * n, &err) : nullptr;
  if (err) { free_all(tmp); return err; }
  r = copy_in(c, dA, A, (size_t)n * n);
  if (!r) {
    eigh_dense(l.ex, l.eig, n, dA, dZ);
    r = launch_status();
  }
  bool sync = false;
  if (!r) r = copy_out(c, w, l.eig.lam, n, &sync);
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

int molgw_b200_tc_gemm(molgw_ctx c, int digits, int M, int N, int K, const double* A, const double* B, double* C) {
  if (!c || M < 1 || N < 1 || K < 1 || !A || !B || !C) return MOLGW_E_ARG;
  if (digits != 0 && digits != 4 && digits != 7) return MOLGW_E_ARG;
  if (digits == 0 && !use_tc(c)) return MOLGW_E_ARG;
  if (digits == 0 && use_fx(c)) digits = kFxSlices;
  DeviceGuard g(c->device);
  Exec& ex = c->lanes[0].ex;
  std::vector<void*> tmp;
  int err = 0;
  double* dA = dalloc(tmp, (size_t)M * K, &err);
  double* dB = dalloc(tmp, (size_t)N * K, &err);
  double* dC = dalloc(tmp, (size_t)M * N, &err);
  if (err) { free_all(tmp); return err; }
  int r = copy_in(c, dA, A, (size_t)M * K);
  if (!r) r = copy_in(c, dB, B, (size_t)N * K);
  if (!r && digits > 0) {
    const long long kp = fx_pad(K);
    const int ns = fx_nsplit((int)kp);
    double* ma = dalloc(tmp, (fx_mat_bytes(M, kp, digits) + 7) / 8, &err);
    double* mb = dalloc(tmp, (fx_mat_bytes(N, kp, digits) + 7) / 8, &err);
    double* part = dalloc(tmp, (size_t)ns * M * N, &err);
    if (err) { free_all(tmp); return err; }
    const FxMat fa = fx_mat_carve(ma, M, kp, digits), fb = fx_mat_carve(mb, N, kp, digits);
    fx_split(ex, dA, M, K, K, 1, nullptr, fa);
    fx_split(ex, dB, N, K, K, 1, nullptr, fb);
    FxGemm gm;
    gm.M = M; gm.N = N; gm.K = (int)kp;
    gm.A = fa; gm.B = fb;
    gm.out = part; gm.out_ld = M; gm.split_stride = (long long)M * N; gm.col_major = true;
    r = fx_gemm(ex, gm);
    if (!r) fx_reduce_cm(ex, part, ns, (long long)M * N, M, N, dC, N, 0.0);
  } else if (!r) {
    const int prec = tc_prec(c);
    const long long kp = tc_pad(K, prec);
    double* ta = dalloc(tmp, (size_t)tc_slices(prec) * (((size_t)M * kp * tc_elem_bytes(prec) + 255) / 256 * 32), &err);
    double* tb = dalloc(tmp, (size_t)tc_slices(prec) * (((size_t)N * kp * tc_elem_bytes(prec) + 255) / 256 * 32), &err);
    const int nkb = (int)(kp / tc_kblock(prec));
    const int ks = tc_ksplit_of(nkb, ceil_div(nkb, std::max(1, 1024 / tc_kblock(prec))));
    float* part = (float*)dalloc(tmp, ((size_t)ks * M * N + 1) / 2, &err);
    if (err) { free_all(tmp); return err; }
    TcMat a, b;
    for (int side = 0; side < 2; ++side) {
      TcMat& t = side ? b : a;
      const long long rows = side ? N : M;
      char* base = (char*)(side ? tb : ta);
      const size_t words = ((size_t)rows * kp * tc_elem_bytes(prec) + 255) / 256 * 256;
      t.rows = rows; t.ld = kp;
      t.hi = base; t.lo = base + words;
      if (tc_slices(prec) == 3) t.lo2 = base + 2 * words;
    }
    tc_split(ex, prec, dA, M, K, K, 1, nullptr, a);
    tc_split(ex, prec, dB, N, K, K, 1, nullptr, b);
    TcGemm gm;
    gm.prec = prec;
    gm.M = M; gm.N = N; gm.K = (int)kp;
    gm.A = a; gm.B = b;
    gm.ksplit = ks;
    gm.epi.mode = TC_EPI_F32_PARTIAL;
    gm.epi.out_f32 = part;
    r = tc_gemm(ex, gm);
    if (!r) tc_reduce_partials(ex, part, ks, M, N, dC, N, 0.0);
  }
  bool sync = false;
  if (!r) r = launch_status();
  if (!r) r = copy_out(c, C, dC, (size_t)M * N, &sync);
  const int st = read_status(c);   // the temporaries are freed below: always synchronise
  free_all(tmp);
  return r ? r : st;
}

int molgw_b200_autotune(molgw_ctx c, int32_t* lanes_out) {
  if (!c) return MOLGW_E_ARG;
  DeviceGuard g(c->device);
  std::vector<int> mols;
  for (int k = 0; k < (int)c->mols.size(); ++k)
    if (ready(c->mols[k])) mols.push_back(k);
  if (mols.empty()) return MOLGW_E_STATE;
  // snapshot of the state a qs_step changes: eps, C, h_MO and the host flags
  std::vector<void*> tmp;
  int err = 0;
  std::vector<double*> snap;
  std::vector<Flags> flags;
  for (int k : mols) {
    const MolBuf& m = c->mols[k];
    const size_t nn = (size_t)m.nb * m.nb, per = m.nb + 2 * nn;
    double* b = dalloc(tmp, m.dn ? 2 * per : per, &err);
    if (err) { free_all(tmp); return err; }
    snap.push_back(b);
    flags.push_back(get_flags(m));
    const MolBuf* chans[2] = {&m, m.dn.get()};
    for (const MolBuf* x : chans) {   // open shell: both spin channels
      if (!x) continue;
      double* bx = (x == &m) ? b : b + per;
      cudaMemcpyAsync(bx, x->eps, m.nb * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
      cudaMemcpyAsync(bx + m.nb, x->C, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
      cudaMemcpyAsync(bx + m.nb + nn, x->hmo, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    }
  }
  auto restore = [&]() {
    for (size_t q = 0; q < mols.size(); ++q) {
      MolBuf& m = c->mols[mols[q]];
      const size_t nn = (size_t)m.nb * m.nb, per = m.nb + 2 * nn;
      MolBuf* chans[2] = {&m, m.dn.get()};
      for (MolBuf* x : chans) {
        if (!x) continue;
        const double* bx = (x == &m) ? snap[q] : snap[q] + per;
        cudaMemcpyAsync(x->eps, bx, m.nb * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(x->C, bx + m.nb, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(x->hmo, bx + m.nb + nn, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
      }
      put_flags(m, flags[q]);
    }
  };
  std::vector<int> cand;
  for (int l : {4, 8, 12, 16}) {
    const int v = std::min(l, (int)mols.size());
    if (cand.empty() || cand.back() != v) cand.push_back(v);
  }
  int best = 0;
  float best_ms = 0.0f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int r = MOLGW_OK;
  {
    // an untimed first trial on one lane measures the tile side of every float64
    // GEMM shape of the pass (the lane trials below then run with those tiles)
    c->tuner.active = true;
    Plan p = plan_batch(c, mols, 1);
    r = plan_fit(c, p);
    if (!r) r = issue_plan(c, p, 'f');
    c->tuner.active = false;
    restore();
    if (!r && cudaStreamSynchronize(c->st) != cudaSuccess) r = cuda_status(cudaGetLastError());
  }
  for (int lanes : cand) {
    if (r) break;
    Plan p = plan_batch(c, mols, lanes);
    r = plan_fit(c, p);
    if (r) break;
    cudaEventRecord(e0, c->st);
    r = issue_plan(c, p, 'f');
    cudaEventRecord(e1, c->st);
    restore();
    if (r) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) { r = cuda_status(cudaGetLastError()); break; }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best == 0 || ms < best_ms) { best = (int)p.lane_mols.size(); best_ms = ms; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int s = read_status(c);   // the snapshot is freed below: synchronise first
  free_all(tmp);
  if (r) return r;
  if (s) return s;
  c->tuned_lanes = best;
  if (lanes_out) *lanes_out = lanes_wanted(c);
  return MOLGW_OK;
}

int32_t molgw_b200_lanes(molgw_ctx c) { return c ? lanes_wanted(c) : 0; }

int molgw_b200_plan_batch(int n_mols, const int32_t* n_basis, const int32_t* n_aux, const int32_t* n_occ_up,
                          const int32_t* n_occ_dn, uint32_t flags, int lanes, int32_t* lane_of, int32_t* slot) {
  if (n_mols < 1 || !n_basis || !n_aux || !n_occ_up || !lane_of || lanes < 0) return MOLGW_E_ARG;
  const bool mp2 = (flags & MOLGW_FLAG_QSMP2) != 0;
  std::vector<double> cost(n_mols);
  for (int k = 0; k < n_mols; ++k) {
    const long long nb = n_basis[k], na = n_aux[k], nu = n_occ_up[k];
    const long long nd = n_occ_dn ? n_occ_dn[k] : -1;
    const bool open = nd >= 0;
    if (nb < 2 || na < 1 || nu < 0 || nu >= nb) return MOLGW_E_ARG;
    if (open ? (nd >= nb || nu + nd < 1 || mp2) : nu < 1) return MOLGW_E_ARG;
    const long long nov = nu * (nb - nu) + (open ? nd * (nb - nd) : 0);
    cost[k] = pass_cost_of(nb, na, nov, open, mp2);
  }
  const auto plan = lpt_assign(cost, std::min(lanes > 0 ? lanes : kDefaultLanes, kMaxLanes));
  for (int j = 0; j < (int)plan.size(); ++j)
    for (int i = 0; i < (int)plan[j].size(); ++i) {
      lane_of[plan[j][i]] = j;
      if (slot) slot[plan[j][i]] = i;
    }
  return (int)plan.size();
}

int64_t molgw_b200_graph_replays(molgw_ctx c) {
  if (!c) return 0;
  return c->graph_off ? -1 : c->graph_replays;
}

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
    for (auto& m : c->mols) { drop_open(m); free_all(m.ri_allocs); free_all(m.orb_allocs); }
    for (auto& t : c->tcb) free_all(t.ri_allocs);
    graph_drop(c);
    for (auto& l : c->lanes) lane_free(l);
    if (c->fork) cudaEventDestroy(c->fork);
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
