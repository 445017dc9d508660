// Host side of the C ABI declared in include/pw.h: problem setup (basis,
// slice geometry, device-resident Fourier tables), the per-k_par eigenmode
// cache, batching of (E, k_par) points and the launch sequence of the sweep.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/pw.h"
#include "pw_internal.h"

using pw::PointDesc;

namespace pw {

const char *kernel_kind_name(int kind) {
  static const char *names[KK_COUNT] = {
      "kb_vectors", "kb_wy ([W|Y] product: kb_wy, kb_wy_tc, kb_wy2_tc or kb_wy2_tc16)", "kb_rowexp",
      "kb_panel", "kb_panel_apply (kb_panel_apply or kb_panel_apply_pair)", "kb_trail (kb_trail or kb_trail_tc)", "kb_rhs_perm", "kb_fsdiag (kb_diag_big<false>)",
      "kb_fsupd_tc", "kb_bsdiag (kb_bsdiag or kb_diag_big<true>)", "kb_bsupd (kb_bsupd or kb_bsupd_tc)",
      "kb_finish",
      "k_refine_init", "k_refine_residual", "k_res_oslice", "k_res_yslice", "k_res_mm", "k_res_finish",
      "k_refine_fwd_a", "k_refine_fwd_b", "k_refine_bwd_a", "k_refine_bwd_b", "k_refine_bwd_mm",
      "k_refine_bwd_c", "k_refine_finish",
      "k_tables", "k_assemble_h", "k_heev (k_heev<double>, or the reduction of k_heev<df>)", "k_ql_df",
      "k_rot_apply", "k_backtransform", "k_eig_sort", "k_overlaps", "k_o32", "k_o32t",
      "k_heev_tail (the FP64 eigensolver's partial last wave on a side stream, beside k_overlaps; its time "
      "includes the wait for free SMs)"};
  return (kind >= 0 && kind < KK_COUNT) ? names[kind] : "";
}

// Launch counts and sampled event pairs of one context (pw_set_profiling).
struct KernelTimer {
  int stride = 1;                      // every stride-th launch of a kind is timed
  long long launches[KK_COUNT] = {};
  long long sampled[KK_COUNT] = {};
  double ms[KK_COUNT] = {};
  struct Rec { cudaEvent_t a, b; int kind; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t take() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // adds the elapsed times of every recorded pair (each waited for) to ms
  cudaError_t flush() {
    cudaError_t first = cudaSuccess;
    for (auto &r : recs) {
      float t = 0.f;
      cudaError_t e = cudaEventSynchronize(r.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
      if (e == cudaSuccess) {
        ms[r.kind] += t;
        sampled[r.kind] += 1;
      } else if (first == cudaSuccess) {
        first = e;
      }
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
    return first;
  }
  void reset() {
    for (int k = 0; k < KK_COUNT; ++k) { launches[k] = 0; sampled[k] = 0; ms[k] = 0.0; }
  }
  ~KernelTimer() {
    for (auto &r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

thread_local KernelTimer *g_ktimer = nullptr;

cudaEvent_t kt_begin(int kind, cudaStream_t s) {
  KernelTimer *t = g_ktimer;
  if (!t || kind < 0 || kind >= KK_COUNT) return nullptr;
  const long long c = t->launches[kind]++;
  if (c % t->stride) return nullptr;
  cudaEvent_t e = t->take();
  if (e) cudaEventRecord(e, s);
  return e;
}

void kt_end(int kind, cudaEvent_t begin, cudaStream_t s) {
  KernelTimer *t = g_ktimer;
  if (!t || !begin) return;
  cudaEvent_t e = t->take();
  if (!e) return;
  cudaEventRecord(e, s);
  t->recs.push_back({begin, e, kind});
}

}  // namespace pw


namespace {

constexpr double kShellQuantum = 1e-8;   // Ry: |G|^2 closer than this is one shell
constexpr double kThreshold = pw::kThresholdRy;
constexpr double kRefineTol = pw::kRefineTolRel;
// default launch variant of the mixed form (pw_set_sweep_variant): the sweep's
// GEMM phases on the tensor cores with the 32-row LU blocks, the refinement
// residual on the CUDA cores in double-float (the measured fastest at
// N_G = 512: 128-row blocks and the slice-product residual were slower), and
// the slice modes and overlaps in FP64: with double-float modes (bit 5, 4x
// faster mode stage) T at the N_G = 512 junction's antiresonance dip
// (T = 0.0036) was 4.8e-8 from the oracle, with FP64 modes 8.8e-10
constexpr int kMixedDefaultVariant = 2;

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct pw_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  pw_status err = PW_OK;
  char err_detail[160] = {0};      // first failing runtime call (pw_get_error_detail)
  int precision = PW_FP64;
  int refine_iters = 0;            // FP64 refinement passes of the mixed form
  int sweep_variant = 0;           // launch variant of the sweep (pw_set_sweep_variant)
  int n = 0, N = 0, nq = 0;        // basis size, slices, slices incl. electrodes
  int Dm = 0, Dn = 0, tsz = 0;     // Fourier-table index ranges
  double b1[2], b2[2], area = 0.0;
  std::vector<int> mn;             // 2n
  std::vector<double> G;           // 2n
  std::vector<double> dz;          // N+2
  int num_sms = 152;
  // device state
  int *d_mn = nullptr;
  double *d_G = nullptr, *d_dz = nullptr, *d_z = nullptr;
  zc *d_tab = nullptr;
  // eigenmode cache: ks_cap k-set slots, each holding the modes of all N+2
  // slices and the N+1 overlaps at one k_par
  int ks_cap = 0;
  std::vector<double> slot_k;      // 2 per slot
  std::vector<char> slot_valid;
  zc *d_HU = nullptr, *d_V = nullptr, *d_O = nullptr;
  cc *d_O32 = nullptr, *d_O32t = nullptr, *d_O32lo = nullptr;   // mixed form: FP32 copies of the
                                                               // overlaps (plain, transposed, remainders)
  double *d_En = nullptr;
  int *d_eigstat = nullptr;       // Jacobi sweeps per matrix
  std::vector<std::vector<double>> EL, ER;   // electrode eigenvalues per slot (host)
  int last_sweeps = 0;                       // most Jacobi sweeps of one matrix in the last eig
  // per-point workspaces
  DevBuf R, M, piv, pts, status, work, KV;
  DevBuf rowexp;                   // row scales of the FP16-split [W|Y] (sweep variant bit 2)
  DevBuf Zst, Ust, LUst, PIVst, Xa, Xb, Fr, Gr, carry, tmp;   // refinement of the mixed form
  DevBuf Xa_m, Xb_m, status_m, Tg, Gam, gtab, T1, dV0, wgt;   // adjoint (pw_grad)
  DevBuf corr;                     // refinement stopping test
  DevBuf eigws;                    // workspace of the double-float eigensolver
  DevBuf bw;                       // batched backward product of the refinement (operands, result)
  int last_passes = 0;             // refinement passes of the last batch
  // device copies of the device-region wells (kept for the adjoint)
  double *d_wxyz = nullptr, *d_wv0 = nullptr, *d_wsig = nullptr;
  int n_wells = 0;
  // transverse motion of the wells and electrodes per unit of the geometry
  // parameter of pw_grad's dgap (2 per well; left, right electrode)
  double *d_wrate = nullptr;
  double lead_rate[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  bool has_shift = false;
  DevBuf dshift, lead_scr, lead_out;
  // launch timing (pw_set_profiling)
  struct Rec { cudaEvent_t a, b; int kind; int count; };
  bool profiling = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> event_pool;
  pw::KernelTimer *kt = nullptr;   // per-kernel launch timing (profiling only)
  int grad_interval = 0;           // pw_grad checkpoint interval (0: ceil(sqrt(N+1)))
  // separable nonlocal projectors (pw_set_projectors)
  int nl_m = 0, nl_q = 0;
  double *d_nlproj = nullptr;      // 6 per projector
  double *d_gl = nullptr;          // Gauss-Legendre nodes, weights
  zc *d_nlD = nullptr;             // m x m
  DevBuf nlV, nlFA, nlFB, nlHA, nlHB, nlPP, ptsb;
  // periodic electrodes (pw_set_periodic_electrode): per side the cell's
  // Fourier tables, slice thicknesses and transverse tilt a3_perp
  int pe_M[2] = {0, 0};
  zc *d_petab[2] = {nullptr, nullptr};
  std::vector<double> pe_dz[2];
  double pe_a3[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  DevBuf peU, peV, peE, peStat, chU, chE, chO, chDz, chPts, chSif, chSa, chSb, chW, chPiv, chSt, bdS[2],
      bdW, bdPiv, bdKeys, bdStates[2], bdProp[2], bdStat, bdE, bdBad, ppW, ppPiv, ppOut;
  DevBuf ckR, ckT;                 // pw_grad checkpoints of the sweep state (R, Tacc)
  // FP64 re-solve of the mixed form's ill-conditioned points (pw_set_fp64_fallback)
  double fb_pivot_max = 1e6, fb_err_max = 1e-8;
  int last_fp64_points = 0;
  double last_pivot_ratio = 0.0;
  DevBuf pivr, R64, M64, piv64, KV64, pts64, st64;
  // second stream and its fork/join events for the two point groups of the
  // sweep (sweep variant bit 6)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // the mode stage's partial wave left running for pw_transmission (ensure_ksets
  // with defer): its stream, the event after its matrices, overlaps and FP32
  // copies, the first interface that needs them, and its matrices' range
  cudaStream_t tail_stream = nullptr, ovl_stream = nullptr;
  cudaEvent_t ev_main = nullptr, ev_tail = nullptr;
  static constexpr int kOvlChunks = 8;
  cudaEvent_t ev_ovl[kOvlChunks] = {};   // after the overlaps (and FP32 copies) of chunk c
  bool tail_pending = false;
  int tail_m0 = 0, tail_m1 = 0;
  int ovl_chunk = 0, ovl_nchunks = 0;     // interfaces per chunk, chunks
};

namespace {

cudaEvent_t take_event(pw_ctx *c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets a stage with events on the context stream when profiling is on.
struct Stage {
  pw_ctx *c;
  cudaEvent_t a = nullptr;
  int kind, count;
  Stage(pw_ctx *ctx, int k, int n) : c(ctx), kind(k), count(n) {
    if (c->profiling) {
      a = take_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  void done() {
    if (!a) return;
    cudaEvent_t b = take_event(c);
    cudaEventRecord(b, c->stream);
    c->recs.push_back({a, b, kind, count});
    a = nullptr;
  }
};

// Interface count C of pw_grad's recomputed segments.
int grad_interval_of(const pw_ctx *c) {
  const int ni = c->N + 1;
  if (c->grad_interval > 0) return std::min(c->grad_interval, ni);
  int C = (int)ceil(sqrt((double)ni));
  return std::max(1, std::min(C, ni));
}

// Installs the context's kernel timer on this host thread for the duration of
// a profiled call (nothing when profiling is off).
struct KtScope {
  pw::KernelTimer *prev;
  explicit KtScope(pw_ctx *c) : prev(pw::g_ktimer) {
    if (c && c->profiling && c->kt) pw::g_ktimer = c->kt;
  }
  ~KtScope() { pw::g_ktimer = prev; }
};

pw_status latch(pw_ctx *c, pw_status s) {
  if (c && c->err == PW_OK && s != PW_OK) c->err = s;
  return s;
}

// The first failing runtime call of a context: its CUDA error and source line.
pw_status latch_cuda(pw_ctx *c, cudaError_t e, int line) {
  if (c && c->err == PW_OK && c->err_detail[0] == 0)
    snprintf(c->err_detail, sizeof(c->err_detail), "%s at pw_api.cu:%d", cudaGetErrorName(e), line);
  return latch(c, e == cudaErrorMemoryAllocation ? PW_ENOMEM : PW_ECUDA);
}

// A failed runtime call is reported once: the runtime's last-error state is
// cleared so that it does not resurface in a later, unrelated call.
#define CK(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      cudaGetLastError();                                                                           \
      return latch_cuda(ctx, e_, __LINE__);                                                         \
    }                                                                                               \
  } while (0)

// With PW_SYNC_CHECK=1 in the environment every stage is followed by a stream
// synchronisation, so that a failing kernel is reported at its own stage.
bool sync_check() {
  static const int on = [] {
    const char *v = getenv("PW_SYNC_CHECK");
    return v && v[0] == '1' ? 1 : 0;
  }();
  return on != 0;
}
#define SYNC_CHECK()                                                                                \
  do {                                                                                              \
    if (sync_check()) CK(cudaStreamSynchronize(ctx->stream));                                       \
  } while (0)

pw_status ensure(pw_ctx *ctx, DevBuf &b, size_t bytes) {
  if (b.bytes >= bytes) return PW_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return latch(ctx, PW_ENOMEM);
  }
  b.bytes = bytes;
  return PW_OK;
}

// Sec. II A: {G = m b1 + n b2}, ordered by (shell, m, n).
void build_basis(const double a1[2], const double a2[2], double ecut, int ng_exact, double b1[2],
                 double b2[2], std::vector<int> &mn, std::vector<double> &G) {
  const double det = a1[0] * a2[1] - a1[1] * a2[0];
  b1[0] = 2.0 * M_PI * a2[1] / det;
  b1[1] = -2.0 * M_PI * a2[0] / det;
  b2[0] = -2.0 * M_PI * a1[1] / det;
  b2[1] = 2.0 * M_PI * a1[0] / det;
  struct Row { long long key; int m, n; double gx, gy; };
  auto enumerate = [&](double ec, std::vector<Row> &rows) {
    rows.clear();
    const double gmax = sqrt(std::max(ec, 0.0));
    const int mmax = (int)floor(gmax * hypot(a1[0], a1[1]) / (2 * M_PI)) + 1;
    const int nmax = (int)floor(gmax * hypot(a2[0], a2[1]) / (2 * M_PI)) + 1;
    for (int m = -mmax; m <= mmax; ++m)
      for (int n = -nmax; n <= nmax; ++n) {
        const double gx = m * b1[0] + n * b2[0], gy = m * b1[1] + n * b2[1];
        const double g2 = gx * gx + gy * gy;
        if (g2 <= ec) rows.push_back({llrint(g2 / kShellQuantum), m, n, gx, gy});
      }
    std::sort(rows.begin(), rows.end(), [](const Row &x, const Row &y) {
      if (x.key != y.key) return x.key < y.key;
      if (x.m != y.m) return x.m < y.m;
      return x.n < y.n;
    });
  };
  std::vector<Row> rows;
  size_t take;
  if (ng_exact > 0) {
    const double amax = std::max(hypot(a1[0], a1[1]), hypot(a2[0], a2[1]));
    double ec = (2 * M_PI) * (2 * M_PI) / (amax * amax);
    for (;;) {
      enumerate(ec, rows);
      if (rows.size() >= (size_t)ng_exact + 64) break;
      ec *= 1.5;
    }
    take = ng_exact;
  } else {
    enumerate(ecut, rows);
    take = rows.size();
  }
  mn.resize(2 * take);
  G.resize(2 * take);
  for (size_t i = 0; i < take; ++i) {
    mn[2 * i] = rows[i].m;
    mn[2 * i + 1] = rows[i].n;
    G[2 * i] = rows[i].gx;
    G[2 * i + 1] = rows[i].gy;
  }
}

template <typename T>
pw_status upload(pw_ctx *ctx, T **dst, const T *src, size_t count) {
  if (count == 0) { *dst = nullptr; return PW_OK; }
  CK(cudaMalloc((void **)dst, count * sizeof(T)));
  CK(cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return PW_OK;
}

// Allocates the k-set slots (as many as fit in a fifth of free memory, <= 4).
pw_status alloc_slots(pw_ctx *ctx) {
  if (ctx->ks_cap) return PW_OK;
  const int n = ctx->n, nq = ctx->nq;
  const size_t nn = (size_t)n * n;
  const bool mixed = ctx->precision == PW_MIXED_FP32;
  const size_t per = (size_t)(3 * nq - 1) * nn * sizeof(zc) + (size_t)nq * n * sizeof(double) +
                     (mixed ? 3 * (size_t)(nq - 1) * nn * sizeof(cc) : 0);
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  int cap = (int)std::min<size_t>(4, std::max<size_t>(1, free_b / 5 / per));
  ctx->ks_cap = cap;
  ctx->slot_k.assign(2 * cap, 0.0);
  ctx->slot_valid.assign(cap, 0);
  ctx->EL.assign(cap, std::vector<double>(n));
  ctx->ER.assign(cap, std::vector<double>(n));
  CK(cudaMalloc(&ctx->d_HU, (size_t)cap * nq * nn * sizeof(zc)));
  CK(cudaMalloc(&ctx->d_V, (size_t)cap * nq * nn * sizeof(zc)));
  CK(cudaMalloc(&ctx->d_O, (size_t)cap * (nq - 1) * nn * sizeof(zc)));
  if (mixed) CK(cudaMalloc(&ctx->d_O32, (size_t)cap * (nq - 1) * nn * sizeof(cc)));
  if (mixed) CK(cudaMalloc(&ctx->d_O32t, (size_t)cap * (nq - 1) * nn * sizeof(cc)));
  if (mixed) CK(cudaMalloc(&ctx->d_O32lo, (size_t)cap * (nq - 1) * nn * sizeof(cc)));
  CK(cudaMalloc(&ctx->d_En, (size_t)cap * nq * n * sizeof(double)));
  CK(cudaMalloc(&ctx->d_eigstat, (size_t)cap * nq * sizeof(int)));
  return PW_OK;
}

// Orders the context's stream after a partial wave left running by
// ensure_ksets (defer) and checks its matrices' convergence.
pw_status join_tail(pw_ctx *ctx) {
  if (!ctx->tail_pending) return PW_OK;
  ctx->tail_pending = false;
  CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_ovl[ctx->ovl_nchunks - 1], 0));
  const int cnt = ctx->tail_m1 - ctx->tail_m0;
  std::vector<int> stat(cnt);
  CK(cudaMemcpyAsync(stat.data(), ctx->d_eigstat + ctx->tail_m0, cnt * sizeof(int), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int v : stat) {
    if (v < 0) {
      ctx->slot_valid.assign(ctx->slot_valid.size(), 0);
      return latch(ctx, PW_ENOTCONV);
    }
  }
  return PW_OK;
}

// Eigenmodes and overlaps of every slice for the k values ks[0..K-1] in slots
// 0..K-1 (K <= ks_cap).  Slots that already hold their k are kept; the others
// are recomputed with one eigensolver launch over all their matrices.
// defer (one slot, FP64 solver): when the solver's grid ends in a partial
// wave, that wave takes the slot's last device slices (the electrodes stay in
// the full waves) and runs on the tail stream, and the overlaps (with their
// FP32 copies) run on the overlap stream in chunks of consecutive interfaces,
// the last ones after the partial wave: on return ctx->tail_pending is set,
// and the caller makes its stream wait for ctx->ev_ovl[c] before interface
// c ctx->ovl_chunk (c < ctx->ovl_nchunks), then calls join_tail.
pw_status ensure_ksets(pw_ctx *ctx, const std::vector<const double *> &ks, bool defer = false) {
  pw_status st = alloc_slots(ctx);
  if (st) return st;
  if ((st = join_tail(ctx))) return st;
  const int n = ctx->n, nq = ctx->nq, K = (int)ks.size();
  const size_t nn = (size_t)n * n;
  int s0 = K, s1 = 0;
  for (int s = 0; s < K; ++s) {
    const bool same = ctx->slot_valid[s] && ctx->slot_k[2 * s] == ks[s][0] &&
                      ctx->slot_k[2 * s + 1] == ks[s][1];
    if (!same) { s0 = std::min(s0, s); s1 = std::max(s1, s + 1); }
  }
  if (s0 >= s1) return PW_OK;
  for (int s = s0; s < s1; ++s) ctx->slot_valid[s] = 0;
  const int nmat = (s1 - s0) * nq;
  Stage st1(ctx, 1, s1 - s0);
  for (int s = s0; s < s1; ++s)
    pw::launch_assemble_h(ctx->d_HU + (size_t)s * nq * nn, ctx->d_tab, ctx->d_mn, ctx->d_G, ks[s][0],
                          ks[s][1], n, nq, ctx->Dm, ctx->Dn, ctx->stream);
  CK(cudaGetLastError());
  // the mixed form's modes and overlaps in FP64, or (variant bit 5) in double-float
  const bool dfe = ctx->precision == PW_MIXED_FP32 && (ctx->sweep_variant & 32);
  if (dfe && (st = ensure(ctx, ctx->eigws, pw::heev_ws_bytes(n, nmat)))) return st;
  zc *HU0 = ctx->d_HU + (size_t)s0 * nq * nn, *V0 = ctx->d_V + (size_t)s0 * nq * nn;
  double *En0 = ctx->d_En + (size_t)s0 * nq * n;
  int *stat0 = ctx->d_eigstat + (size_t)s0 * nq;
  // The FP64 solver runs one matrix per CTA.  When its grid ends in a partial
  // wave, that wave's matrices go to a side stream, and the overlaps of every
  // interface whose two slices are in the full waves run beside it on the SMs
  // the partial wave leaves idle; the remaining overlaps follow both.
  int nA = nmat;
  if (!dfe) {
    const int res = pw::heev_resident_per_sm(n) * ctx->num_sms;
    if (res > 0 && nmat > res && nmat % res) nA = nmat - nmat % res;
  }
  if (defer && !dfe && s1 - s0 == 1 && nA < nmat && nA >= 3) {
    // the partial wave beside the sweep: matrices nA-1 .. nq-2 (device slices)
    // on the tail stream; the full waves take 0 .. nA-2 and the right
    // electrode nq-1 (the grid's last CTA)
    if (!ctx->tail_stream) {
      bool ok = cudaStreamCreateWithFlags(&ctx->tail_stream, cudaStreamNonBlocking) == cudaSuccess &&
                cudaStreamCreateWithFlags(&ctx->ovl_stream, cudaStreamNonBlocking) == cudaSuccess &&
                cudaEventCreateWithFlags(&ctx->ev_main, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&ctx->ev_tail, cudaEventDisableTiming) == cudaSuccess;
      for (int c = 0; ok && c < pw_ctx::kOvlChunks; ++c)
        ok = cudaEventCreateWithFlags(&ctx->ev_ovl[c], cudaEventDisableTiming) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        return latch(ctx, PW_ECUDA);
      }
    }
    cudaStream_t ts = ctx->tail_stream, os = ctx->ovl_stream;
    zc *O0 = ctx->d_O + (size_t)s0 * (nq - 1) * nn;
    const int gT = nA - 2;   // pairs g < gT use the full waves' slices only
    CK(cudaEventRecord(ctx->ev_main, ctx->stream));   // the Hamiltonians are assembled
    CK(cudaStreamWaitEvent(ts, ctx->ev_main, 0));
    pw::launch_eig(HU0, V0, En0, stat0, n, nA, ctx->stream, false, nullptr, 0, false, nq - 1);
    pw::launch_eig(HU0 + (size_t)(nA - 1) * nn, V0 + (size_t)(nA - 1) * nn, En0 + (size_t)(nA - 1) * n,
                   stat0 + (nA - 1), n, nmat - nA, ts, false, nullptr, 0, true);
    CK(cudaEventRecord(ctx->ev_tail, ts));
    CK(cudaGetLastError());
    CK(cudaEventRecord(ctx->ev_main, ctx->stream));   // the full waves' modes (and the right electrode's)
    st1.done();
    // overlaps in chunks on the overlap stream, beside the sweep: interface p
    // needs only O_p (and the modes of slices p, p+1)
    const int npairs = nq - 1, nch = std::min(pw_ctx::kOvlChunks, npairs);
    const int L = (npairs + nch - 1) / nch;
    CK(cudaStreamWaitEvent(os, ctx->ev_main, 0));
    bool waited_tail = false;
    int c = 0;
    for (int g0 = 0; g0 < npairs; g0 += L, ++c) {
      const int g1 = std::min(npairs, g0 + L);
      if (g1 > gT && !waited_tail) {   // pairs from gT on need the partial wave's slices
        CK(cudaStreamWaitEvent(os, ctx->ev_tail, 0));
        waited_tail = true;
      }
      pw::launch_overlaps(HU0, O0, n, nq, 1, os, false, g0, g1);
      if (ctx->d_O32)
        pw::launch_overlaps_fp32(O0 + (size_t)g0 * nn, ctx->d_O32 + ((size_t)s0 * (nq - 1) + g0) * nn,
                                 ctx->d_O32t + ((size_t)s0 * (nq - 1) + g0) * nn,
                                 ctx->d_O32lo + ((size_t)s0 * (nq - 1) + g0) * nn, n, g1 - g0, os);
      CK(cudaEventRecord(ctx->ev_ovl[c], os));
    }
    CK(cudaGetLastError());
    // the full waves' convergence and the electrodes' eigenvalues now; the
    // partial wave's convergence in join_tail
    std::vector<int> stat(nA);
    CK(cudaMemcpyAsync(stat.data(), stat0, (nA - 1) * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(stat.data() + nA - 1, stat0 + nq - 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->EL[s0].data(), En0, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->ER[s0].data(), En0 + (size_t)(nq - 1) * n, n * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->last_sweeps = 0;
    for (int v : stat) {
      if (v < 0) {
        CK(cudaStreamSynchronize(os));
        return latch(ctx, PW_ENOTCONV);
      }
      ctx->last_sweeps = std::max(ctx->last_sweeps, v);
    }
    ctx->tail_pending = true;
    ctx->ovl_chunk = L;
    ctx->ovl_nchunks = c;
    ctx->tail_m0 = s0 * nq + nA - 1;
    ctx->tail_m1 = s0 * nq + nq - 1;
    ctx->slot_k[2 * s0] = ks[s0][0];
    ctx->slot_k[2 * s0 + 1] = ks[s0][1];
    ctx->slot_valid[s0] = 1;
    return PW_OK;
  }
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  if (nA < nmat) {
    if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();   // no side stream: one launch
      if (side) cudaStreamDestroy(side);
      if (fork) cudaEventDestroy(fork);
      side = nullptr;
      fork = nullptr;
      nA = nmat;
    } else {
      CK(cudaEventRecord(fork, ctx->stream));
      CK(cudaStreamWaitEvent(side, fork, 0));
    }
  }
  pw::launch_eig(HU0, V0, En0, stat0, n, nA, ctx->stream, dfe, dfe ? ctx->eigws.p : nullptr,
                 dfe ? ctx->eigws.bytes : 0);
  if (side)
    pw::launch_eig(HU0 + (size_t)nA * nn, V0 + (size_t)nA * nn, En0 + (size_t)nA * n, stat0 + nA, n, nmat - nA,
                   side, false, nullptr, 0, true);
  CK(cudaGetLastError());
  SYNC_CHECK();
  st1.done();
  Stage st2(ctx, 2, s1 - s0);
  const int npairs = (s1 - s0) * (nq - 1);
  int gA = 0;   // pairs g < gA have both slices among the first nA matrices
  while (gA < npairs && (gA / (nq - 1)) * nq + gA % (nq - 1) + 1 < nA) ++gA;
  pw::launch_overlaps(HU0, ctx->d_O + (size_t)s0 * (nq - 1) * nn, n, nq, s1 - s0, ctx->stream, dfe, 0, gA);
  if (side) {
    CK(cudaEventRecord(join, side));
    CK(cudaStreamWaitEvent(ctx->stream, join, 0));
    cudaEventDestroy(fork);
    cudaEventDestroy(join);
    cudaStreamDestroy(side);
  }
  pw::launch_overlaps(HU0, ctx->d_O + (size_t)s0 * (nq - 1) * nn, n, nq, s1 - s0, ctx->stream, dfe, gA, npairs);
  if (ctx->d_O32)
    pw::launch_overlaps_fp32(ctx->d_O + (size_t)s0 * (nq - 1) * nn, ctx->d_O32 + (size_t)s0 * (nq - 1) * nn,
                             ctx->d_O32t + (size_t)s0 * (nq - 1) * nn, ctx->d_O32lo + (size_t)s0 * (nq - 1) * nn,
                             n, (s1 - s0) * (nq - 1), ctx->stream);
  CK(cudaGetLastError());
  SYNC_CHECK();
  st2.done();
  std::vector<int> stat(nmat);
  CK(cudaMemcpyAsync(stat.data(), ctx->d_eigstat + (size_t)s0 * nq, nmat * sizeof(int),
                     cudaMemcpyDeviceToHost, ctx->stream));
  for (int s = s0; s < s1; ++s) {
    CK(cudaMemcpyAsync(ctx->EL[s].data(), ctx->d_En + (size_t)s * nq * n, n * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->ER[s].data(), ctx->d_En + ((size_t)s * nq + nq - 1) * n,
                       n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->last_sweeps = 0;
  for (int i = 0; i < nmat; ++i) {
    if (stat[i] < 0) return latch(ctx, PW_ENOTCONV);
    ctx->last_sweeps = std::max(ctx->last_sweeps, stat[i]);
  }
  for (int s = s0; s < s1; ++s) {
    ctx->slot_k[2 * s] = ks[s][0];
    ctx->slot_k[2 * s + 1] = ks[s][1];
    ctx->slot_valid[s] = 1;
  }
  return PW_OK;
}

pw_status ensure_kset(pw_ctx *ctx, const double *k) {
  return ensure_ksets(ctx, std::vector<const double *>{k});
}

int count_open(const std::vector<double> &En, double E, bool *thresh) {
  int c = 0;
  for (double v : En) {
    if (fabs(E - v) < kThreshold) *thresh = true;
    if (v < E) ++c;
  }
  return c;
}

// Unique k values in first-appearance order and the points of each.
void group_by_k(int npts, const double *kpar, std::vector<std::vector<int>> &groups) {
  groups.clear();
  std::vector<std::pair<double, double>> keys;
  for (int i = 0; i < npts; ++i) {
    const std::pair<double, double> k(kpar[2 * i], kpar[2 * i + 1]);
    size_t g = 0;
    for (; g < keys.size(); ++g)
      if (keys[g] == k) break;
    if (g == keys.size()) {
      keys.push_back(k);
      groups.emplace_back();
    }
    groups[g].push_back(i);
  }
}

}  // namespace

pw::CtxView pw::ctx_view(const pw_ctx *c) {
  CtxView v;
  v.n = c->n;
  v.N = c->N;
  v.Dm = c->Dm;
  v.Dn = c->Dn;
  v.num_sms = c->num_sms;
  v.precision = c->precision;
  v.refine_iters = c->refine_iters;
  v.tab = c->d_tab;
  v.mn = c->d_mn;
  v.G = c->d_G;
  v.dz = c->dz.data();
  v.stream = c->stream;
  return v;
}

extern "C" {

const char *pw_status_str(pw_status s) {
  switch (s) {
    case PW_OK: return "ok";
    case PW_EINVAL: return "invalid argument";
    case PW_ENOMEM: return "device allocation failed";
    case PW_ECUDA: return "CUDA runtime error";
    case PW_ESINGULAR: return "zero pivot in LU factorisation";
    case PW_ETHRESH: return "energy at an electrode channel threshold";
    case PW_ETIMEOUT: return "bounded device wait timed out";
    case PW_ENOTCONV: return "eigensolver did not converge";
  }
  return "unknown status";
}

pw_status pw_get_error(const pw_ctx *ctx) { return ctx ? ctx->err : PW_EINVAL; }
pw_status pw_get_error_detail(const pw_ctx *ctx, char *buf, int len) {
  if (!ctx || !buf || len <= 0) return PW_EINVAL;
  snprintf(buf, (size_t)len, "%s", ctx->err_detail);
  return PW_OK;
}
int pw_ng(const pw_ctx *ctx) { return ctx ? ctx->n : 0; }
int pw_n_slices(const pw_ctx *ctx) { return ctx ? ctx->N : 0; }

pw_status pw_get_gvectors(const pw_ctx *ctx, int *mn_host) {
  if (!ctx || !mn_host) return PW_EINVAL;
  memcpy(mn_host, ctx->mn.data(), ctx->mn.size() * sizeof(int));
  return PW_OK;
}

pw_status pw_setup(const pw_setup_desc *d, void *cuda_stream, pw_ctx **out) {
  if (!d || !out) return PW_EINVAL;
  *out = nullptr;
  if (d->n_slices < 1 || !d->z_edges) return PW_EINVAL;
  if (d->precision != PW_FP64 && d->precision != PW_MIXED_FP32) return PW_EINVAL;
  for (int i = 0; i < d->n_slices; ++i)
    if (!(d->z_edges[i + 1] > d->z_edges[i])) return PW_EINVAL;
  if (!d->slice_vg && d->n_wells > 0 && (!d->well_xyz || !d->well_v0 || !d->well_sigma))
    return PW_EINVAL;
  for (int s = 0; s < 2; ++s)
    if (!d->lead_vg[s] && d->lead_n_wells[s] > 0 &&
        (!d->lead_well_xy[s] || !d->lead_well_v0[s] || !d->lead_well_sigma[s] || !(d->lead_period[s] > 0)))
      return PW_EINVAL;
  const double det = d->a1[0] * d->a2[1] - d->a1[1] * d->a2[0];
  if (!(fabs(det) > 0)) return PW_EINVAL;
  pw_ctx *ctx = new (std::nothrow) pw_ctx();
  if (!ctx) return PW_ENOMEM;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->precision = d->precision;
  if (d->refine_iters < -1 || d->refine_iters > 16) { delete ctx; return PW_EINVAL; }
  ctx->refine_iters = d->precision == PW_MIXED_FP32 ? (d->refine_iters == 0 ? 4 : std::max(0, d->refine_iters)) : 0;
  ctx->sweep_variant = d->precision == PW_MIXED_FP32 ? kMixedDefaultVariant : 0;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) { delete ctx; return PW_ECUDA; }
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  build_basis(d->a1, d->a2, d->ecut, d->ng_exact, ctx->b1, ctx->b2, ctx->mn, ctx->G);
  ctx->n = (int)(ctx->mn.size() / 2);
  if (ctx->n < 1 || ctx->n > 1024) { delete ctx; return PW_EINVAL; }
  ctx->N = d->n_slices;
  ctx->nq = ctx->N + 2;
  ctx->area = fabs(det);
  int mmax = 0, nmax = 0;
  for (int i = 0; i < ctx->n; ++i) {
    mmax = std::max(mmax, abs(ctx->mn[2 * i]));
    nmax = std::max(nmax, abs(ctx->mn[2 * i + 1]));
  }
  ctx->Dm = 2 * mmax;
  ctx->Dn = 2 * nmax;
  ctx->tsz = (2 * ctx->Dm + 1) * (2 * ctx->Dn + 1);
  if (d->slice_vg || d->lead_vg[0] || d->lead_vg[1]) {
    if (d->vg_half[0] < 0 || d->vg_half[1] < 0) { delete ctx; return PW_EINVAL; }
  }
  ctx->dz.assign(ctx->nq, 0.0);
  for (int p = 1; p <= ctx->N; ++p) ctx->dz[p] = d->z_edges[p] - d->z_edges[p - 1];
  pw_status st;
  if ((st = upload(ctx, &ctx->d_mn, ctx->mn.data(), ctx->mn.size())) != PW_OK ||
      (st = upload(ctx, &ctx->d_G, ctx->G.data(), ctx->G.size())) != PW_OK ||
      (st = upload(ctx, &ctx->d_dz, ctx->dz.data(), ctx->dz.size())) != PW_OK ||
      (st = upload(ctx, &ctx->d_z, d->z_edges, (size_t)ctx->N + 1)) != PW_OK) {
    pw_destroy(ctx);
    return st;
  }
  // Fourier tables: explicit ones are embedded on the host, wells on the device
  const size_t tab_bytes = (size_t)ctx->nq * ctx->tsz * sizeof(zc);
  if (cudaMalloc(&ctx->d_tab, tab_bytes) != cudaSuccess) { pw_destroy(ctx); return PW_ENOMEM; }
  std::vector<zc> host_tab;
  auto embed = [&](const pw_c128 *src, int q) {
    const int sm = d->vg_half[0], sn = d->vg_half[1];
    zc *dst = host_tab.data() + (size_t)q * ctx->tsz;
    for (int i = -std::min(sm, ctx->Dm); i <= std::min(sm, ctx->Dm); ++i)
      for (int j = -std::min(sn, ctx->Dn); j <= std::min(sn, ctx->Dn); ++j) {
        const pw_c128 v = src[(size_t)(i + sm) * (2 * sn + 1) + (j + sn)];
        dst[(size_t)(i + ctx->Dm) * (2 * ctx->Dn + 1) + (j + ctx->Dn)] = mkc<double>(v.re, v.im);
      }
  };
  const bool any_explicit = d->slice_vg || d->lead_vg[0] || d->lead_vg[1];
  if (any_explicit) {
    host_tab.assign((size_t)ctx->nq * ctx->tsz, mkc<double>(0.0, 0.0));
    if (d->slice_vg) {
      const size_t stride = (size_t)(2 * d->vg_half[0] + 1) * (2 * d->vg_half[1] + 1);
      for (int p = 1; p <= ctx->N; ++p) embed(d->slice_vg + (p - 1) * stride, p);
    }
    if (d->lead_vg[0]) embed(d->lead_vg[0], 0);
    if (d->lead_vg[1]) embed(d->lead_vg[1], ctx->nq - 1);
    if (cudaMemcpyAsync(ctx->d_tab, host_tab.data(), tab_bytes, cudaMemcpyHostToDevice, ctx->stream) !=
        cudaSuccess) { pw_destroy(ctx); return PW_ECUDA; }
  }
  pw::TableArgs ta;
  memset(&ta, 0, sizeof(ta));
  ta.tab = ctx->d_tab;
  ta.nq = ctx->nq;
  ta.Dm = ctx->Dm;
  ta.Dn = ctx->Dn;
  ta.b1x = ctx->b1[0]; ta.b1y = ctx->b1[1]; ta.b2x = ctx->b2[0]; ta.b2y = ctx->b2[1];
  ta.area = ctx->area;
  ta.z_edges = ctx->d_z;
  ta.explicit_slices = d->slice_vg ? 1 : 0;
  ta.explicit_lead[0] = d->lead_vg[0] ? 1 : 0;
  ta.explicit_lead[1] = d->lead_vg[1] ? 1 : 0;
  std::vector<void *> temps;
  auto up = [&](const double *src, size_t cnt) -> const double * {
    if (!src || cnt == 0) return nullptr;
    double *p = nullptr;
    if (upload(ctx, &p, src, cnt) != PW_OK) return nullptr;
    temps.push_back(p);
    return p;
  };
  if (!d->slice_vg && d->n_wells > 0) {
    if ((st = upload(ctx, &ctx->d_wxyz, d->well_xyz, 3 * (size_t)d->n_wells)) != PW_OK ||
        (st = upload(ctx, &ctx->d_wv0, d->well_v0, (size_t)d->n_wells)) != PW_OK ||
        (st = upload(ctx, &ctx->d_wsig, d->well_sigma, (size_t)d->n_wells)) != PW_OK) {
      pw_destroy(ctx);
      return st;
    }
    ctx->n_wells = d->n_wells;
    if (d->well_shift_rate) {
      if ((st = upload(ctx, &ctx->d_wrate, d->well_shift_rate, 2 * (size_t)d->n_wells)) != PW_OK) {
        pw_destroy(ctx);
        return st;
      }
      ctx->has_shift = true;
    }
    ta.slices.xyz = ctx->d_wxyz;
    ta.slices.v0 = ctx->d_wv0;
    ta.slices.sigma = ctx->d_wsig;
    ta.slices.n = d->n_wells;
  }
  for (int s = 0; s < 2; ++s)
    for (int c = 0; c < 2; ++c) {
      ctx->lead_rate[s][c] = d->lead_shift_rate[s][c];
      if (d->lead_shift_rate[s][c] != 0.0) ctx->has_shift = true;
    }
  for (int s = 0; s < 2; ++s) {
    ta.period[s] = d->lead_period[s] > 0 ? d->lead_period[s] : 1.0;
    if (!d->lead_vg[s] && d->lead_n_wells[s] > 0) {
      ta.lead[s].xyz = up(d->lead_well_xy[s], 2 * (size_t)d->lead_n_wells[s]);
      ta.lead[s].v0 = up(d->lead_well_v0[s], d->lead_n_wells[s]);
      ta.lead[s].sigma = up(d->lead_well_sigma[s], d->lead_n_wells[s]);
      ta.lead[s].n = d->lead_n_wells[s];
    }
  }
  if (ctx->err != PW_OK) { st = ctx->err; pw_destroy(ctx); return st; }
  pw::launch_tables(ta, ctx->stream);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  for (void *p : temps) cudaFree(p);
  if (e != cudaSuccess) { pw_destroy(ctx); return PW_ECUDA; }
  *out = ctx;
  return PW_OK;
}

void pw_destroy(pw_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->side) {
    cudaStreamSynchronize(ctx->side);
    cudaStreamDestroy(ctx->side);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  for (cudaStream_t t : {ctx->tail_stream, ctx->ovl_stream}) {
    if (t) {
      cudaStreamSynchronize(t);
      cudaStreamDestroy(t);
    }
  }
  if (ctx->ev_main) cudaEventDestroy(ctx->ev_main);
  if (ctx->ev_tail) cudaEventDestroy(ctx->ev_tail);
  for (cudaEvent_t e : ctx->ev_ovl)
    if (e) cudaEventDestroy(e);
  void *bufs[] = {ctx->d_mn, ctx->d_G, ctx->d_dz, ctx->d_z, ctx->d_tab, ctx->d_HU, ctx->d_V,
                  ctx->d_O, ctx->d_O32, ctx->d_O32t, ctx->d_O32lo, ctx->d_En, ctx->d_eigstat, ctx->R.p, ctx->M.p, ctx->piv.p,
                  ctx->pts.p, ctx->status.p, ctx->work.p, ctx->KV.p, ctx->Zst.p, ctx->Ust.p, ctx->Xa.p,
                  ctx->Xb.p, ctx->Fr.p, ctx->Gr.p, ctx->carry.p, ctx->tmp.p, ctx->LUst.p,
                  ctx->PIVst.p, ctx->Xa_m.p, ctx->Xb_m.p, ctx->status_m.p, ctx->Tg.p, ctx->Gam.p,
                  ctx->gtab.p, ctx->T1.p, ctx->dV0.p, ctx->wgt.p, ctx->d_wxyz, ctx->d_wv0,
                  ctx->d_wsig, ctx->corr.p, ctx->d_wrate, ctx->dshift.p, ctx->lead_scr.p,
                  ctx->lead_out.p, ctx->eigws.p, ctx->bw.p, ctx->rowexp.p, ctx->ckR.p, ctx->ckT.p,
                  ctx->d_nlproj, ctx->d_gl, ctx->d_nlD, ctx->nlV.p, ctx->nlFA.p, ctx->nlFB.p, ctx->nlHA.p,
                  ctx->nlHB.p, ctx->nlPP.p, ctx->ptsb.p, ctx->d_petab[0], ctx->d_petab[1], ctx->peU.p,
                  ctx->peV.p, ctx->peE.p, ctx->peStat.p, ctx->chU.p, ctx->chE.p, ctx->chO.p, ctx->chDz.p,
                  ctx->chPts.p, ctx->chSif.p, ctx->chSa.p, ctx->chSb.p, ctx->chW.p, ctx->chPiv.p, ctx->chSt.p,
                  ctx->bdS[0].p, ctx->bdS[1].p, ctx->bdW.p, ctx->bdPiv.p, ctx->bdKeys.p, ctx->bdStates[0].p,
                  ctx->bdStates[1].p, ctx->bdProp[0].p, ctx->bdProp[1].p, ctx->bdStat.p, ctx->bdE.p,
                  ctx->bdBad.p, ctx->ppW.p, ctx->ppPiv.p, ctx->ppOut.p};
  for (void *p : bufs)
    if (p) cudaFree(p);
  for (auto &r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  delete ctx->kt;
  delete ctx;
}

pw_status pw_set_sweep_variant(pw_ctx *ctx, int variant) {
  if (!ctx || variant < 0 || variant >= pw::sweep_variants(ctx->precision)) return PW_EINVAL;
  ctx->sweep_variant = variant;
  return PW_OK;
}

pw_status pw_set_profiling(pw_ctx *ctx, int enable) {
  if (!ctx || enable < 0) return PW_EINVAL;
  ctx->profiling = enable != 0;
  if (enable) {
    if (!ctx->kt) ctx->kt = new (std::nothrow) pw::KernelTimer;
    if (!ctx->kt) return PW_ENOMEM;
    ctx->kt->stride = enable;
  }
  return PW_OK;
}

int pw_kernel_kinds(void) { return pw::KK_COUNT; }

const char *pw_kernel_kind_name(int kind) { return pw::kernel_kind_name(kind); }

pw_status pw_eig_wave(int n, int *matrices) {
  if (n < 1 || !matrices) return PW_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return PW_ECUDA;
  }
  *matrices = pw::heev_resident_per_sm(n) * sms;
  return PW_OK;
}

pw_status pw_get_kernel_profile(pw_ctx *ctx, double *out, int reset) {
  if (!ctx || !out) return PW_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < pw::KK_COUNT; ++k) out[3 * k] = out[3 * k + 1] = out[3 * k + 2] = 0.0;
  if (!ctx->kt) return PW_OK;
  CK(ctx->kt->flush());
  for (int k = 0; k < pw::KK_COUNT; ++k) {
    out[3 * k] = ctx->kt->ms[k];
    out[3 * k + 1] = (double)ctx->kt->sampled[k];
    out[3 * k + 2] = (double)ctx->kt->launches[k];
  }
  if (reset) ctx->kt->reset();
  return PW_OK;
}

pw_status pw_get_profile(pw_ctx *ctx, double *out, int reset) {
  if (!ctx || !out) return PW_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < 10; ++i) out[i] = 0.0;
  for (auto &r : ctx->recs) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    out[2 * r.kind] += ms;
    out[2 * r.kind + 1] += r.count;
  }
  if (reset) {
    for (auto &r : ctx->recs) { ctx->event_pool.push_back(r.a); ctx->event_pool.push_back(r.b); }
    ctx->recs.clear();
  }
  return PW_OK;
}

pw_status pw_potential_tables(pw_ctx *ctx, pw_c128 *vg_dev, int *half_host) {
  if (!ctx) return PW_EINVAL;
  if (ctx->err) return ctx->err;
  if (half_host) { half_host[0] = ctx->Dm; half_host[1] = ctx->Dn; }
  if (vg_dev)
    CK(cudaMemcpyAsync(vg_dev, ctx->d_tab, (size_t)ctx->nq * ctx->tsz * sizeof(zc),
                       cudaMemcpyDeviceToDevice, ctx->stream));
  return PW_OK;
}

pw_status pw_slice_modes(pw_ctx *ctx, const double *kpar, double *En_dev, pw_c128 *U_dev) {
  if (!ctx || !kpar) return PW_EINVAL;
  if (ctx->err) return ctx->err;
  pw_status st = ensure_kset(ctx, kpar);
  if (st) return st;
  const size_t nn = (size_t)ctx->n * ctx->n;
  if (En_dev)
    CK(cudaMemcpyAsync(En_dev, ctx->d_En, (size_t)ctx->nq * ctx->n * sizeof(double),
                       cudaMemcpyDeviceToDevice, ctx->stream));
  if (U_dev)
    CK(cudaMemcpyAsync(U_dev, ctx->d_HU, ctx->nq * nn * sizeof(zc), cudaMemcpyDeviceToDevice,
                       ctx->stream));
  return PW_OK;
}

pw_status pw_overlaps(pw_ctx *ctx, const double *kpar, pw_c128 *O_dev) {
  if (!ctx || !kpar || !O_dev) return PW_EINVAL;
  if (ctx->err) return ctx->err;
  pw_status st = ensure_kset(ctx, kpar);
  if (st) return st;
  CK(cudaMemcpyAsync(O_dev, ctx->d_O, (size_t)(ctx->nq - 1) * ctx->n * ctx->n * sizeof(zc),
                     cudaMemcpyDeviceToDevice, ctx->stream));
  return PW_OK;
}

pw_status slice_blocks(pw_ctx *ctx, int npts, const double *E, const double *kpar, int iface, pw_c128 *S_dev,
                       int mixed);

pw_status pw_slice_smatrix(pw_ctx *ctx, int npts, const double *E, const double *kpar, int iface,
                           pw_c128 *S_dev) {
  return slice_blocks(ctx, npts, E, kpar, iface, S_dev, 0);
}

pw_status pw_slice_mixed(pw_ctx *ctx, int npts, const double *E, const double *kpar, int iface,
                         pw_c128 *T_dev) {
  return slice_blocks(ctx, npts, E, kpar, iface, T_dev, 1);
}

pw_status slice_blocks(pw_ctx *ctx, int npts, const double *E, const double *kpar, int iface, pw_c128 *S_dev,
                       int mixed) {
  if (!ctx || npts < 0 || (npts > 0 && (!E || !kpar || !S_dev))) return PW_EINVAL;
  if (ctx->err) return ctx->err;
  if (iface < 0 || iface > ctx->N) return PW_EINVAL;
  const int n = ctx->n;
  const size_t nn = (size_t)n * n;
  std::vector<std::vector<int>> groups;
  group_by_k(npts, kpar, groups);
  for (auto &g : groups) {
    pw_status st = ensure_kset(ctx, kpar + 2 * g[0]);
    if (st) return st;
    const int bmax = std::max(1, std::min((int)g.size(), 2 * ctx->num_sms));
    for (size_t b0 = 0; b0 < g.size(); b0 += bmax) {
      const int nb = (int)std::min(g.size() - b0, (size_t)bmax);
      if ((st = ensure(ctx, ctx->work, (size_t)nb * 3 * nn * sizeof(zc))) ||
          (st = ensure(ctx, ctx->piv, (size_t)nb * n * sizeof(int))) ||
          (st = ensure(ctx, ctx->pts, (size_t)nb * sizeof(PointDesc))) ||
          (st = ensure(ctx, ctx->status, (size_t)nb * sizeof(int))) ||
          (st = ensure(ctx, ctx->M, (size_t)nb * 4 * nn * sizeof(zc))))
        return st;
      std::vector<PointDesc> pd(nb);
      for (int i = 0; i < nb; ++i) {
        const int idx = g[b0 + i];
        pd[i] = pw::make_point(E[idx], 0, 0, 0, idx, 0, ctx->N, i);
      }
      CK(cudaMemcpyAsync(ctx->pts.p, pd.data(), nb * sizeof(PointDesc), cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemsetAsync(ctx->status.p, 0, nb * sizeof(int), ctx->stream));
      CK(pw::launch_slice_smatrix((PointDesc *)ctx->pts.p, ctx->d_En, ctx->d_O, ctx->d_dz,
                                  (zc *)ctx->work.p, (int *)ctx->piv.p, (int *)ctx->status.p,
                                  (zc *)ctx->M.p, n, ctx->N, iface, nb, ctx->stream, mixed));
      // scatter the batch's S blocks to the caller's point order
      for (int i = 0; i < nb; ++i)
        CK(cudaMemcpyAsync(S_dev + (size_t)g[b0 + i] * 4 * nn, (zc *)ctx->M.p + (size_t)i * 4 * nn,
                           4 * nn * sizeof(zc), cudaMemcpyDeviceToDevice, ctx->stream));
      std::vector<int> st_h(nb);
      CK(cudaMemcpyAsync(st_h.data(), ctx->status.p, nb * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      for (int v : st_h)
        if (v) return latch(ctx, PW_ESINGULAR);
    }
  }
  return PW_OK;
}

pw_status pw_compose(pw_ctx *ctx, int npts, const pw_c128 *Sa_dev, const pw_c128 *Sb_dev,
                     pw_c128 *Sab_dev) {
  if (!ctx || npts < 0 || (npts > 0 && (!Sa_dev || !Sb_dev || !Sab_dev))) return PW_EINVAL;
  if (ctx->err) return ctx->err;
  const int n = ctx->n;
  const size_t nn = (size_t)n * n;
  const int bmax = std::max(1, std::min(npts, 2 * ctx->num_sms));
  pw_status st;
  for (int b0 = 0; b0 < npts; b0 += bmax) {
    const int nb = std::min(npts - b0, bmax);
    if ((st = ensure(ctx, ctx->work, (size_t)nb * 4 * nn * sizeof(zc))) ||
        (st = ensure(ctx, ctx->piv, (size_t)nb * n * sizeof(int))) ||
        (st = ensure(ctx, ctx->status, (size_t)nb * sizeof(int))))
      return st;
    CK(cudaMemsetAsync(ctx->status.p, 0, nb * sizeof(int), ctx->stream));
    CK(pw::launch_compose((const zc *)Sa_dev + (size_t)b0 * 4 * nn, (const zc *)Sb_dev + (size_t)b0 * 4 * nn,
                          (zc *)Sab_dev + (size_t)b0 * 4 * nn, (zc *)ctx->work.p, (int *)ctx->piv.p,
                          (int *)ctx->status.p, n, nb, ctx->stream));
    std::vector<int> st_h(nb);
    CK(cudaMemcpyAsync(st_h.data(), ctx->status.p, nb * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int v : st_h)
      if (v) return latch(ctx, PW_ESINGULAR);
  }
  return PW_OK;
}

pw_status pw_compose_mixed(pw_ctx *ctx, int npts, const pw_c128 *Ta_dev, const pw_c128 *Tb_dev,
                           pw_c128 *Tab_dev) {
  if (!ctx || npts < 0 || (npts > 0 && (!Ta_dev || !Tb_dev || !Tab_dev))) return PW_EINVAL;
  if (ctx->err) return ctx->err;
  const int n = ctx->n;
  const size_t nn = (size_t)n * n;
  const int bmax = std::max(1, std::min(npts, 2 * ctx->num_sms));
  const pw::Strides str{4 * nn, 4 * nn, 4 * nn};
  pw_status st;
  for (int b0 = 0; b0 < npts; b0 += bmax) {
    const int nb = std::min(npts - b0, bmax);
    if ((st = ensure(ctx, ctx->work, (size_t)nb * 4 * nn * sizeof(zc))) ||
        (st = ensure(ctx, ctx->piv, (size_t)nb * n * sizeof(int))) ||
        (st = ensure(ctx, ctx->status, (size_t)nb * sizeof(int))))
      return st;
    CK(cudaMemsetAsync(ctx->status.p, 0, nb * sizeof(int), ctx->stream));
    CK(pw::launch_compose_mixed((const zc *)Ta_dev + (size_t)b0 * 4 * nn, (const zc *)Tb_dev + (size_t)b0 * 4 * nn,
                                (zc *)Tab_dev + (size_t)b0 * 4 * nn, (zc *)ctx->work.p, (int *)ctx->piv.p,
                                (int *)ctx->status.p, n, nb, ctx->stream, str));
    std::vector<int> st_h(nb);
    CK(cudaMemcpyAsync(st_h.data(), ctx->status.p, nb * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int v : st_h)
      if (v) return latch(ctx, PW_ESINGULAR);
  }
  return PW_OK;
}

// Layer doubling of one point's interface elements (FP64), one point at a
// time: A holds the N+1 mixed elements, B half as many; each level combines
// neighbours from one into the other (an odd last block is copied up).
pw_status pw_transmission_doubling(pw_ctx *ctx, int npts, const double *E, const double *kpar,
                                   double cond_max, double *T_dev, int *levels_host) {
  if (!ctx || npts < 0 || (npts > 0 && (!E || !kpar || !T_dev)) || !(cond_max > 0.0)) return PW_EINVAL;
  if (ctx->err) return ctx->err;
  KtScope kts(ctx);
  const int n = ctx->n, N = ctx->N, nblk = N + 1;
  const size_t nn = (size_t)n * n, blk = 4 * nn;
  const int cap = std::max(1, 2 * ctx->num_sms);   // CTAs per launch (bounds the work buffers)
  std::vector<std::vector<int>> groups;
  group_by_k(npts, kpar, groups);
  pw_status result = PW_OK, st;
  if ((st = alloc_slots(ctx))) return st;
  DevBuf &A = ctx->M, &B = ctx->R;
  if ((st = ensure(ctx, A, (size_t)nblk * blk * sizeof(zc))) ||
      (st = ensure(ctx, B, (size_t)((nblk + 1) / 2) * blk * sizeof(zc))) ||
      (st = ensure(ctx, ctx->work, (size_t)std::min(cap, nblk) * blk * sizeof(zc))) ||
      (st = ensure(ctx, ctx->piv, (size_t)std::min(cap, nblk) * n * sizeof(int))) ||
      (st = ensure(ctx, ctx->status, (size_t)std::min(cap, nblk) * sizeof(int))) ||
      (st = ensure(ctx, ctx->corr, (size_t)nblk * sizeof(double))) ||
      (st = ensure(ctx, ctx->pts, sizeof(PointDesc))))
    return st;
  int *stat = (int *)ctx->status.p;
  int *piv = (int *)ctx->piv.p;
  zc *work = (zc *)ctx->work.p;
  double *norms = (double *)ctx->corr.p;
  auto check_status = [&](int count) -> pw_status {
    std::vector<int> h(count);
    CK(cudaMemcpyAsync(h.data(), stat, count * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int v : h)
      if (v) return latch(ctx, PW_ESINGULAR);
    return PW_OK;
  };
  auto max_norm = [&](const zc *T, int count, double *out) -> pw_status {
    CK(pw::launch_i11_norm(T, blk, n, count, norms, ctx->stream));
    std::vector<double> h(count);
    CK(cudaMemcpyAsync(h.data(), norms, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *out = 0.0;
    for (double v : h) *out = std::max(*out, v);
    return PW_OK;
  };
  auto to_s = [&](zc *T, int count) -> pw_status {
    for (int b0 = 0; b0 < count; b0 += cap) {
      const int nb = std::min(count - b0, cap);
      CK(cudaMemsetAsync(stat, 0, nb * sizeof(int), ctx->stream));
      CK(pw::launch_mixed_to_s(T + (size_t)b0 * blk, blk, work, piv, stat, n, nb, ctx->stream));
      pw_status s2 = check_status(nb);
      if (s2) return s2;
    }
    return PW_OK;
  };
  const double nan = std::nan("");
  for (auto &g : groups) {
    if ((st = ensure_kset(ctx, kpar + 2 * g[0]))) return st;
    for (int idx : g) {
      bool th = false;
      const int nL = count_open(ctx->EL[0], E[idx], &th);
      const int nR = count_open(ctx->ER[0], E[idx], &th);
      if (levels_host) levels_host[idx] = -1;
      if (th) {
        result = PW_ETHRESH;
        CK(cudaMemcpyAsync(T_dev + idx, &nan, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        continue;
      }
      const PointDesc pd = pw::make_point(E[idx], 0, nL, nR, idx, 0, N, 0);
      CK(cudaMemcpyAsync(ctx->pts.p, &pd, sizeof(PointDesc), cudaMemcpyHostToDevice, ctx->stream));
      // the mixed elements of every interface, cap interfaces per launch
      for (int f0 = 0; f0 < nblk; f0 += cap) {
        const int nb = std::min(nblk - f0, cap);
        CK(cudaMemsetAsync(stat, 0, nb * sizeof(int), ctx->stream));
        CK(pw::launch_slice_smatrix((PointDesc *)ctx->pts.p, ctx->d_En, ctx->d_O, ctx->d_dz, work, piv, stat,
                                    (zc *)A.p + (size_t)f0 * blk, n, N, f0, nb, ctx->stream, 1, blk, 1));
        if ((st = check_status(nb))) return st;
      }
      zc *src = (zc *)A.p, *dst = (zc *)B.p;
      int cnt = nblk, level = 0;
      double g_max = 0.0;
      if ((st = max_norm(src, cnt, &g_max))) return st;
      bool mixed = g_max <= cond_max;
      if (!mixed && (st = to_s(src, cnt))) return st;
      while (cnt > 1) {
        const int pairs = cnt / 2;
        for (int i0 = 0; i0 < pairs; i0 += cap) {
          const int nb = std::min(pairs - i0, cap);
          const pw::Strides str{2 * blk, 2 * blk, blk};
          const zc *a = src + (size_t)2 * i0 * blk, *b = a + blk;
          zc *c = dst + (size_t)i0 * blk;
          CK(cudaMemsetAsync(stat, 0, nb * sizeof(int), ctx->stream));
          if (mixed) CK(pw::launch_compose_mixed(a, b, c, work, piv, stat, n, nb, ctx->stream, str));
          else CK(pw::launch_compose(a, b, c, work, piv, stat, n, nb, ctx->stream, str));
          if ((st = check_status(nb))) return st;
        }
        if (cnt & 1)
          CK(cudaMemcpyAsync(dst + (size_t)pairs * blk, src + (size_t)(cnt - 1) * blk, blk * sizeof(zc),
                             cudaMemcpyDeviceToDevice, ctx->stream));
        cnt = pairs + (cnt & 1);
        std::swap(src, dst);
        if (mixed) {
          ++level;
          if ((st = max_norm(src, cnt, &g_max))) return st;
          if (g_max > cond_max) {
            mixed = false;
            if ((st = to_s(src, cnt))) return st;
          }
        }
      }
      if (mixed && (st = to_s(src, 1))) return st;
      const double *EnL = ctx->d_En, *EnR = ctx->d_En + (size_t)(N + 1) * n;
      CK(pw::launch_t_from_s(src, EnL, EnR, E[idx], n, nL, nR, T_dev + idx, ctx->stream));
      if (levels_host) levels_host[idx] = level;
    }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return result;
}

// The FP64 sweep (every interface in FP64, from the FP64 modes and overlaps
// of the points' k-set slots) of the points pts, writing their T, t, n_open
// and a zero error estimate; status_out[i] is point i's sweep status.
static pw_status fp64_sweep(pw_ctx *ctx, std::vector<PointDesc> pts, int nc, double *T_dev, pw_c128 *t_dev,
                            int *nopen_dev, double *err_dev, std::vector<int> &status_out) {
  const int n = ctx->n, N = ctx->N, ncols = 2 * n + nc;
  const size_t nn = (size_t)n * n, esz = sizeof(zc);
  status_out.assign(pts.size(), 0);
  const int cap = std::max(1, 2 * ctx->num_sms);
  pw_status st = PW_OK;
  for (size_t b0 = 0; b0 < pts.size(); b0 += cap) {
    const int nb = (int)std::min(pts.size() - b0, (size_t)cap);
    std::vector<PointDesc> pd(pts.begin() + b0, pts.begin() + b0 + nb);
    for (int i = 0; i < nb; ++i)
      pd[i] = pw::make_point(pd[i].E, pd[i].kset, pd[i].nL, pd[i].nR, pd[i].out, 0, N, i);
    if ((st = ensure(ctx, ctx->R64, (size_t)nb * nn * esz)) ||
        (st = ensure(ctx, ctx->M64, (size_t)nb * n * ncols * esz)) ||
        (st = ensure(ctx, ctx->piv64, (size_t)nb * n * sizeof(int))) ||
        (st = ensure(ctx, ctx->KV64, (size_t)nb * 3 * n * esz)) ||
        (st = ensure(ctx, ctx->pts64, (size_t)nb * sizeof(PointDesc))) ||
        (st = ensure(ctx, ctx->st64, (size_t)nb * sizeof(int))))
      return st;
    CK(cudaMemcpyAsync(ctx->pts64.p, pd.data(), nb * sizeof(PointDesc), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->st64.p, 0, nb * sizeof(int), ctx->stream));
    pw::SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.pts = (const PointDesc *)ctx->pts64.p;
    a.En = ctx->d_En;
    a.O = ctx->d_O;
    a.dz = ctx->d_dz;
    a.R = ctx->R64.p;
    a.M = ctx->M64.p;
    a.piv = (int *)ctx->piv64.p;
    a.status = (int *)ctx->st64.p;
    a.T = T_dev;
    a.t = (zc *)t_dev;
    a.nopen = nopen_dev;
    a.err = err_dev;
    a.n = n;
    a.N = N;
    a.nc = nc;
    a.KV = ctx->KV64.p;
    CK(pw::prepare_sweep_batched(n, PW_FP64, 0));
    for (int p = 0; p <= N; ++p) {
      CK(pw::launch_sweep_batched(a, nb, p, PW_FP64, ctx->stream, nullptr, nullptr, 0));
      SYNC_CHECK();
    }
    CK(cudaMemcpyAsync(status_out.data() + b0, ctx->st64.p, nb * sizeof(int), cudaMemcpyDeviceToHost,
                       ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return PW_OK;
}

// The mixed form's FP64 fallback for one batch after its sweep and refinement
// (pd: the batch's descriptors; status: the FP32 sweep's per-point status,
// updated for the points solved again).  A point is solved again by the FP64
// sweep when an LU factor of some W_p has a diagonal spread max|u_ii| /
// min|u_ii| above fb_pivot_max (then W_p's condition number is at least that
// large), when its estimated error after the last refinement pass is above
// fb_err_max, or when the FP32 sweep met a zero pivot.
static pw_status fp64_fallback(pw_ctx *ctx, const std::vector<PointDesc> &pd, int nc, std::vector<int> &status,
                               double *T_dev, pw_c128 *t_dev, int *nopen_dev, double *err_dev) {
  const int nb = (int)pd.size();
  if (ctx->fb_pivot_max < 0.0) return PW_OK;
  std::vector<float> pr(nb);
  std::vector<double> cr(2 * (size_t)nb);
  CK(cudaMemcpyAsync(pr.data(), ctx->pivr.p, nb * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(cr.data(), ctx->corr.p, 2 * (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<PointDesc> redo;
  std::vector<int> which;
  for (int i = 0; i < nb; ++i) {
    if (pd[i].skip || status[i] == 2) continue;   // threshold point; a timed-out wait stays an error
    const double c = cr[i], cp = cr[nb + i];
    const double est = cp > 0.0 ? c * c / cp : c;   // the refinement's own estimate
    if (status[i] == 0) ctx->last_pivot_ratio = std::max(ctx->last_pivot_ratio, (double)pr[i]);
    if (status[i] == 1 || !((double)pr[i] <= ctx->fb_pivot_max) || !(est <= ctx->fb_err_max)) {
      redo.push_back(pd[i]);
      which.push_back(i);
    }
  }
  if (redo.empty()) return PW_OK;
  std::vector<int> st64;
  pw_status st = fp64_sweep(ctx, redo, nc, T_dev, t_dev, nopen_dev, err_dev, st64);
  if (st) return st;
  for (size_t j = 0; j < which.size(); ++j) status[which[j]] = st64[j];
  ctx->last_fp64_points += (int)redo.size();
  return PW_OK;
}

pw_status pw_set_fp64_fallback(pw_ctx *ctx, double pivot_ratio_max, double err_max) {
  if (!ctx || pivot_ratio_max != pivot_ratio_max || !(err_max >= 0.0)) return PW_EINVAL;
  ctx->fb_pivot_max = pivot_ratio_max;
  ctx->fb_err_max = err_max;
  return PW_OK;
}

pw_status pw_get_fp64_fallback(const pw_ctx *ctx, int *points, double *max_pivot_ratio) {
  if (!ctx || !points || !max_pivot_ratio) return PW_EINVAL;
  *points = ctx->last_fp64_points;
  *max_pivot_ratio = ctx->last_pivot_ratio;
  return PW_OK;
}

pw_status pw_transmission(pw_ctx *ctx, int npts, const double *E, const double *kpar, double *T_dev,
                          pw_c128 *t_dev, int *nopen_dev, double *err_dev) {
  if (!ctx || npts < 0 || (npts > 0 && (!E || !kpar || !T_dev))) return PW_EINVAL;
  if (ctx->err) return ctx->err;
  KtScope kts(ctx);
  const int n = ctx->n;
  const size_t nn = (size_t)n * n;
  const size_t esz = ctx->precision == PW_FP64 ? sizeof(zc) : sizeof(cc);
  std::vector<std::vector<int>> groups;
  group_by_k(npts, kpar, groups);
  pw_status result = PW_OK;
  pw_status st = alloc_slots(ctx);
  if (st) return st;
  ctx->last_fp64_points = 0;
  ctx->last_pivot_ratio = 0.0;
  for (size_t g0 = 0; g0 < groups.size(); g0 += ctx->ks_cap) {
    const size_t g1 = std::min(groups.size(), g0 + (size_t)ctx->ks_cap);
    std::vector<const double *> ks;
    std::vector<std::pair<int, int>> pts;   // (point index, slot)
    for (size_t gi = g0; gi < g1; ++gi) {
      ks.push_back(kpar + 2 * groups[gi][0]);
      for (int idx : groups[gi]) pts.emplace_back(idx, (int)(gi - g0));
    }
    // one k_par: the eigensolver's partial wave and the overlaps run beside
    // the first interfaces of the sweep (which waits for each chunk of them)
    if ((st = ensure_ksets(ctx, ks, ks.size() == 1))) return st;
    // point descriptors and the padded incident-column count of the chunk
    std::vector<PointDesc> all(pts.size());
    int nc = 1;
    for (size_t i = 0; i < pts.size(); ++i) {
      const int idx = pts[i].first, slot = pts[i].second;
      bool th = false;
      const int nL = count_open(ctx->EL[slot], E[idx], &th);
      const int nR = count_open(ctx->ER[slot], E[idx], &th);
      all[i] = pw::make_point(E[idx], slot, nL, nR, idx, th ? 1 : 0, ctx->N, 0);
      if (th) result = PW_ETHRESH;
      else nc = std::max(nc, nL);
    }
    nc = (nc + 3) & ~3;
    const int ncols = 2 * n + nc;
    const int N = ctx->N;
    const bool refine = ctx->precision == PW_MIXED_FP32 && ctx->refine_iters > 0;
    // per-point bytes of the sweep (+ refinement) buffers; the batch fits in 85 %
    // of the free memory
    size_t per_pt = nn * esz + (size_t)n * ncols * esz + 3 * (size_t)n * esz + n * sizeof(int) + 64;
    if (refine)
      per_pt += (size_t)(N + 1) * (2 * nn + (size_t)n * nc) * sizeof(cc) + (size_t)(N + 1) * n * sizeof(int) +
                (size_t)(2 * (N + 2) + 2 * (N + 1) + 1) * n * nc * sizeof(zc) + 2 * (size_t)n * nc * sizeof(cc);
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const size_t have = free_b + ctx->R.bytes + ctx->M.bytes + ctx->Zst.bytes + ctx->Ust.bytes +
                        ctx->LUst.bytes + ctx->PIVst.bytes +
                        ctx->Xa.bytes + ctx->Xb.bytes + ctx->Fr.bytes + ctx->Gr.bytes;
    const int fit = (int)std::max<size_t>(1, (size_t)(0.85 * (double)have) / per_pt);
    const int bmax = std::max(1, std::min({(int)pts.size(), 3 * ctx->num_sms, fit}));
    for (size_t b0 = 0; b0 < pts.size(); b0 += bmax) {
      const int nb = (int)std::min(pts.size() - b0, (size_t)bmax);
      std::vector<PointDesc> pd(all.begin() + b0, all.begin() + b0 + nb);
      for (int i = 0; i < nb; ++i) pd[i] = pw::make_point(pd[i].E, pd[i].kset, pd[i].nL, pd[i].nR, pd[i].out,
                                                          pd[i].skip, N, i);
      if ((st = ensure(ctx, ctx->R, (size_t)nb * nn * esz)) ||
          (st = ensure(ctx, ctx->M, (size_t)nb * n * ncols * esz)) ||
          (st = ensure(ctx, ctx->piv, (size_t)nb * n * sizeof(int))) ||
          (st = ensure(ctx, ctx->KV, (size_t)nb * 3 * n * esz)) ||
          (st = ensure(ctx, ctx->pts, (size_t)nb * sizeof(PointDesc))) ||
          (st = ensure(ctx, ctx->status, (size_t)nb * sizeof(int))) ||
          ((ctx->sweep_variant & 4) && (st = ensure(ctx, ctx->rowexp, (size_t)nb * 2 * n * sizeof(int)))))
        return st;
      const size_t vec = (size_t)nb * n * nc;
      if (refine &&
          ((st = ensure(ctx, ctx->Zst, (size_t)nb * (N + 1) * nn * sizeof(cc))) ||
           (st = ensure(ctx, ctx->LUst, (size_t)nb * (N + 1) * nn * sizeof(cc))) ||
           (st = ensure(ctx, ctx->PIVst, (size_t)nb * (N + 1) * n * sizeof(int))) ||
           (st = ensure(ctx, ctx->Ust, (size_t)(N + 1) * vec * sizeof(cc))) ||
           (st = ensure(ctx, ctx->Xa, (size_t)(N + 2) * vec * sizeof(zc))) ||
           (st = ensure(ctx, ctx->Xb, (size_t)(N + 2) * vec * sizeof(zc))) ||
           (st = ensure(ctx, ctx->Fr, (size_t)(N + 1) * vec * sizeof(zc))) ||
           (st = ensure(ctx, ctx->Gr, (size_t)(N + 1) * vec * sizeof(zc))) ||
           (st = ensure(ctx, ctx->carry, vec * sizeof(zc))) ||
           (st = ensure(ctx, ctx->corr, (size_t)2 * nb * sizeof(double))) ||
           (st = ensure(ctx, ctx->tmp, 2 * vec * sizeof(cc)))))
        return st;
      CK(cudaMemcpyAsync(ctx->pts.p, pd.data(), nb * sizeof(PointDesc), cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemsetAsync(ctx->status.p, 0, nb * sizeof(int), ctx->stream));
      pw::SweepArgs a;
      memset(&a, 0, sizeof(a));
      a.pts = (const PointDesc *)ctx->pts.p;
      a.En = ctx->d_En;
      a.O = ctx->d_O;
      a.O32 = ctx->d_O32;
      a.O32t = ctx->d_O32t;
      a.dz = ctx->d_dz;
      a.R = ctx->R.p;
      a.M = ctx->M.p;
      a.piv = (int *)ctx->piv.p;
      a.status = (int *)ctx->status.p;
      a.T = T_dev;
      a.t = refine ? nullptr : (zc *)t_dev;
      a.nopen = nopen_dev;
      a.err = err_dev;
      a.n = n;
      a.N = N;
      a.nc = nc;
      a.Zst = refine ? ctx->Zst.p : nullptr;
      a.Ust = refine ? ctx->Ust.p : nullptr;
      a.LUst = refine ? ctx->LUst.p : nullptr;
      a.PIVst = refine ? (int *)ctx->PIVst.p : nullptr;
      a.KV = ctx->KV.p;
      a.mirror = 0;
      a.wy_pairs = pw::points_pair_up(pd.data(), nb);
      a.rowexp = (ctx->sweep_variant & 4) ? (int *)ctx->rowexp.p : nullptr;
      if (refine) {
        if ((st = ensure(ctx, ctx->pivr, (size_t)nb * sizeof(float)))) return st;
        CK(cudaMemsetAsync(ctx->pivr.p, 0, nb * sizeof(float), ctx->stream));
        a.pivratio = (float *)ctx->pivr.p;
      }
      CK(pw::prepare_sweep_batched(n, ctx->precision, ctx->sweep_variant));
      // the FP16-split [W|Y] adds its row-scale kernel at every interface with a product (p >= 1)
      const int f16_extra = (a.rowexp && a.wy_pairs && (ctx->sweep_variant & 6) == 6) ? N : 0;
      // Sweep variant bit 6: the batch as two point groups, each swept on its
      // own stream, so that one group's latency-bound kernels (panels,
      // diagonal blocks, one CTA per point) run beside the other group's
      // wide update kernels.  The groups share no per-point state.
      int hA = nb;
      cudaStream_t s2 = nullptr;
      if ((ctx->sweep_variant & 64) && nb >= 32) {
        hA = (nb / 2) & ~1;
        if (!ctx->side) {
          if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
              cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
              cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return latch(ctx, PW_ECUDA);
          }
        }
        s2 = ctx->side;
      }
      pw::SweepArgs aB = a;
      if (s2) {
        a.wy_pairs = pw::points_pair_up(pd.data(), hA);
        aB.wy_pairs = pw::points_pair_up(pd.data() + hA, nb - hA);
        aB.pts = a.pts + hA;
        aB.R = (unsigned char *)a.R + (size_t)hA * nn * esz;
        aB.M = (unsigned char *)a.M + (size_t)hA * n * ncols * esz;
        aB.piv = a.piv + (size_t)hA * n;
        aB.status = a.status + hA;
        aB.KV = (unsigned char *)a.KV + (size_t)hA * 3 * n * esz;
        if (a.rowexp) aB.rowexp = a.rowexp + (size_t)hA * 2 * n;
        if (a.pivratio) aB.pivratio = a.pivratio + hA;
        CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
        CK(cudaStreamWaitEvent(s2, ctx->ev_fork, 0));
      }
      Stage s0(ctx, 0, (s2 ? 2 : 1) * (N + 1) * pw::sweep_batched_launches(n, ctx->precision, ctx->sweep_variant) +
                           f16_extra);
      for (int p = 0; p <= N; ++p) {
        if (ctx->tail_pending && p % ctx->ovl_chunk == 0 && p / ctx->ovl_chunk < ctx->ovl_nchunks) {
          // the overlaps of interfaces p .. p + ovl_chunk - 1 (and the partial
          // wave's modes they need) are ready after this chunk's event
          const cudaEvent_t e = ctx->ev_ovl[p / ctx->ovl_chunk];
          CK(cudaStreamWaitEvent(ctx->stream, e, 0));
          if (s2) CK(cudaStreamWaitEvent(s2, e, 0));
        }
        cudaEvent_t w0 = nullptr, w1 = nullptr;
        if (ctx->profiling && p > 0) { w0 = take_event(ctx); w1 = take_event(ctx); }
        CK(pw::launch_sweep_batched(a, hA, p, ctx->precision, ctx->stream, w0, w1, ctx->sweep_variant));
        if (w0) ctx->recs.push_back({w0, w1, 4, 1});
        if (s2) CK(pw::launch_sweep_batched(aB, nb - hA, p, ctx->precision, s2, nullptr, nullptr, ctx->sweep_variant));
        SYNC_CHECK();
      }
      if (s2) {
        CK(cudaEventRecord(ctx->ev_join, s2));
        CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
      }
      s0.done();
      if (refine) {
        pw::RefineArgs r;
        memset(&r, 0, sizeof(r));
        r.pts = a.pts;
        r.En = a.En;
        r.O = a.O;
        r.O32 = a.O32;
        r.O32lo = ctx->d_O32lo;
        r.dz = a.dz;
        r.Zst = (const cc *)ctx->Zst.p;
        r.Ust = (cc *)ctx->Ust.p;
        r.LUst = (const cc *)ctx->LUst.p;
        r.PIVst = (const int *)ctx->PIVst.p;
        r.M = (cc *)ctx->M.p;
        r.piv = a.piv;
        r.status = a.status;
        r.Xa = (zc *)ctx->Xa.p;
        r.Xb = (zc *)ctx->Xb.p;
        r.Fr = (zc *)ctx->Fr.p;
        r.Gr = (zc *)ctx->Gr.p;
        r.carry = (zc *)ctx->carry.p;
        r.tmp = (cc *)ctx->tmp.p;
        r.corr = (double *)ctx->corr.p;
        r.corr_prev = r.corr + nb;
        r.T = T_dev;
        r.t = (zc *)t_dev;
        r.nopen = nopen_dev;
        r.err = err_dev;
        r.n = n;
        r.N = N;
        r.nc = nc;
        r.x_slots = (long long)nb * (N + 2);
        r.st_slots = (long long)nb * (N + 1);
        r.piv_order = pw::stored_piv_order(ctx->sweep_variant);   // the stored factors' pivot order
        if (pw::points_share_overlaps(pd.data(), nb) && ctx->d_O32) {
          // one buffer: the backward product's operands and result, then (when the
          // residual runs on the tensor cores) O y, the slices and their exponents
          auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
          const long long ncol = 2LL * nb * nc;
          const bool sliced = (ctx->sweep_variant & 16) && ctx->d_O32lo && n <= 512 && n % 4 == 0;
          const size_t b_bw = up((size_t)4 * nb * n * nc * sizeof(cc));
          const size_t b_y = up((size_t)2 * n * ncol * sizeof(double));
          const size_t b_sl = up(pw::rs_slice_bytes(n, ncol));
          const size_t b_ex = ((size_t)2 * n + ncol) * sizeof(int);
          if ((st = ensure(ctx, ctx->bw, b_bw + (sliced ? b_y + b_sl + b_ex : 0))) == PW_OK) {
            unsigned char *base = (unsigned char *)ctx->bw.p;
            r.Bw = (cc *)base;
            r.Yw = r.Bw + (size_t)2 * nb * n * nc;
            if (sliced) {
              r.Yacc = (double *)(base + b_bw);
              r.Osl = (uint16_t *)(base + b_bw + b_y);
              r.Ysl = r.Osl + (size_t)pw::RS_SLICES * 4 * n * n;
              r.Oexp = (int *)(base + b_bw + b_y + b_sl);
              r.Yexp = r.Oexp + 2 * n;
            }
          }
        }
        if (st) return st;
        Stage s3(ctx, 3, 1);
        int passes = 0;
        CK(pw::launch_refine(r, nb, std::min(2, ctx->refine_iters), ctx->refine_iters, kRefineTol,
                             ctx->stream, &passes));
        SYNC_CHECK();
        s3.count = passes;
        s3.done();
        ctx->last_passes = passes;
      }
      std::vector<int> st_h(nb);
      CK(cudaMemcpyAsync(st_h.data(), ctx->status.p, nb * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      if (ctx->profiling && ctx->kt) CK(ctx->kt->flush());   // keeps the pending event pairs bounded
      if (refine && (st = fp64_fallback(ctx, pd, nc, st_h, T_dev, t_dev, nopen_dev, err_dev))) return st;
      for (int v : st_h) {
        if (v == 2) result = PW_ETIMEOUT;   // a tensor-core wait ran out (kept over a zero pivot)
        else if (v && result != PW_ETIMEOUT) result = PW_ESINGULAR;
      }
    }
    if ((st = join_tail(ctx))) return st;
  }
  if (result == PW_ESINGULAR || result == PW_ETIMEOUT) latch(ctx, result);
  return result;
}


// The FP64 sweep of a batch of nb points with its stores (Z_p, u_p) and the
// backward pass that recovers every slice's amplitudes into g.Xa, g.Xb, in
// segments of C interfaces: with K > 1 segments a first pass keeps only the
// sweep state (R and the Tacc columns) before every segment after the first;
// the segments are then taken from the right, each recomputed with its stores
// (slots st_off + p = i C + p - p0 of point i) and stepped through backward
// (the carry links consecutive segments).  loc / d_loc: the points' host and
// device descriptors (their st_off is rewritten per segment).
static pw_status stored_sweep_backward(pw_ctx *ctx, const pw::SweepArgs &a, const pw::GradArgs &g, int nb, int C,
                                       std::vector<PointDesc> &loc, PointDesc *d_loc) {
  const int n = ctx->n, N = ctx->N, ncols = 2 * n + a.nc;
  const size_t nn = (size_t)n * n, vec = (size_t)n * a.nc;
  const int K = (N + 1 + C - 1) / C;
  CK(pw::prepare_sweep_batched(n, PW_FP64, 0));
  zc *Rb = (zc *)ctx->R.p, *Mb = (zc *)ctx->M.p;
  zc *ckR = (zc *)ctx->ckR.p, *ckT = (zc *)ctx->ckT.p;
  if (K > 1) {
    pw::SweepArgs a0 = a;
    a0.Zst = nullptr;
    a0.Ust = nullptr;
    for (int p = 0; p <= N; ++p) {
      CK(pw::launch_sweep_batched(a0, nb, p, PW_FP64, ctx->stream));
      if ((p + 1) % C == 0 && p < N) {
        const int k = (p + 1) / C - 1;
        CK(cudaMemcpyAsync(ckR + (size_t)k * nb * nn, Rb, (size_t)nb * nn * sizeof(zc), cudaMemcpyDeviceToDevice,
                           ctx->stream));
        CK(cudaMemcpy2DAsync(ckT + (size_t)k * nb * vec, vec * sizeof(zc), Mb + 2 * nn, (size_t)n * ncols * sizeof(zc),
                             vec * sizeof(zc), nb, cudaMemcpyDeviceToDevice, ctx->stream));
      }
    }
  }
  for (int k = K - 1; k >= 0; --k) {
    const int p0 = k * C, p1 = std::min(N, p0 + C - 1);
    for (int i = 0; i < nb; ++i) loc[i].st_off = (long long)i * C - p0;
    CK(cudaMemcpyAsync(d_loc, loc.data(), nb * sizeof(PointDesc), cudaMemcpyHostToDevice, ctx->stream));
    if (k > 0) {
      CK(cudaMemcpyAsync(Rb, ckR + (size_t)(k - 1) * nb * nn, (size_t)nb * nn * sizeof(zc), cudaMemcpyDeviceToDevice,
                         ctx->stream));
      CK(cudaMemcpy2DAsync(Mb + 2 * nn, (size_t)n * ncols * sizeof(zc), ckT + (size_t)(k - 1) * nb * vec,
                           vec * sizeof(zc), vec * sizeof(zc), nb, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    for (int p = p0; p <= p1; ++p) CK(pw::launch_sweep_batched(a, nb, p, PW_FP64, ctx->stream));
    CK(pw::launch_grad_backward(g, nb, ctx->stream, p1, p0, k == K - 1));
  }
  return PW_OK;
}

// Gauss-Legendre nodes x[q] and weights w[q] on [-1, 1]: Newton iteration on
// the Legendre polynomial P_q from the Chebyshev-like first guesses
// cos(pi (i + 3/4) / (q + 1/2)), P_q and P_q' by the three-term recurrence.
static void gauss_legendre(int q, double *x, double *w) {
  for (int i = 0; i < q; ++i) {
    double z = cos(M_PI * (i + 0.75) / (q + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= q; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double pq = q == 1 ? z : p1, pm = q == 1 ? 1.0 : p0;
      dp = q * (z * pq - pm) / (z * z - 1.0);
      const double dz = pq / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[q - 1 - i] = z;
    w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

pw_status pw_set_projectors(pw_ctx *ctx, int m, const double *params, const pw_c128 *D, int quad_nodes) {
  if (!ctx || m < 0 || m > pw::kNlMaxProj || (m > 0 && (!params || !D)) || quad_nodes < 2 ||
      quad_nodes > pw::kNlMaxQuad)
    return PW_EINVAL;
  if (ctx->err) return ctx->err;
  for (int a = 0; a < m; ++a)
    if (!(params[6 * a + 3] > 0.0) || !(params[6 * a + 4] <= params[6 * a + 5])) return PW_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  for (void **b : {(void **)&ctx->d_nlproj, (void **)&ctx->d_gl, (void **)&ctx->d_nlD})
    if (*b) { cudaFree(*b); *b = nullptr; }
  ctx->nl_m = 0;
  if (m == 0) return PW_OK;
  std::vector<double> gl(2 * quad_nodes);
  gauss_legendre(quad_nodes, gl.data(), gl.data() + quad_nodes);
  if (cudaMalloc(&ctx->d_nlproj, 6 * m * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_gl, gl.size() * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_nlD, (size_t)m * m * sizeof(zc)) != cudaSuccess) {
    cudaGetLastError();
    return latch(ctx, PW_ENOMEM);
  }
  CK(cudaMemcpy(ctx->d_nlproj, params, 6 * m * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_gl, gl.data(), gl.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_nlD, D, (size_t)m * m * sizeof(zc), cudaMemcpyHostToDevice));
  ctx->nl_m = m;
  ctx->nl_q = quad_nodes;
  return PW_OK;
}

pw_status pw_transmission_nonlocal(pw_ctx *ctx, int npts, const double *E, const double *kpar, double *T_dev,
                                   pw_c128 *C_dev) {
  if (!ctx || npts < 0 || (npts > 0 && (!E || !kpar || !T_dev)) || ctx->nl_m <= 0) return PW_EINVAL;
  if (ctx->err) return ctx->err;
  KtScope kts(ctx);
  const int n = ctx->n, N = ctx->N, m = ctx->nl_m;
  const size_t nn = (size_t)n * n;
  pw_status st = alloc_slots(ctx);
  if (st) return st;
  std::vector<std::vector<int>> groups;
  group_by_k(npts, kpar, groups);
  pw_status result = PW_OK;
  const int C = grad_interval_of(ctx);
  const int K = (N + 1 + C - 1) / C;
  for (size_t g0 = 0; g0 < groups.size(); g0 += ctx->ks_cap) {
    const size_t g1 = std::min(groups.size(), g0 + (size_t)ctx->ks_cap);
    std::vector<const double *> ks;
    std::vector<std::pair<int, int>> pts;
    for (size_t gi = g0; gi < g1; ++gi) {
      ks.push_back(kpar + 2 * groups[gi][0]);
      for (int idx : groups[gi]) pts.emplace_back(idx, (int)(gi - g0));
    }
    if ((st = ensure_ksets(ctx, ks))) return st;
    // the projectors in every device slice's mode basis, per k-set
    if ((st = ensure(ctx, ctx->nlV, (size_t)ks.size() * N * m * n * sizeof(zc)))) return st;
    for (size_t sl = 0; sl < ks.size(); ++sl)
      CK(pw::launch_nl_project(ctx->d_HU + sl * (size_t)(N + 2) * nn, (zc *)ctx->nlV.p + sl * (size_t)N * m * n,
                               nullptr, ctx->d_G, ks[sl][0], ks[sl][1], ctx->d_nlproj, ctx->area, n, N, m,
                               ctx->stream));
    std::vector<PointDesc> all(pts.size());
    int ninc = 1;
    for (size_t i = 0; i < pts.size(); ++i) {
      const int idx = pts[i].first, slot = pts[i].second;
      bool th = false;
      const int nL = count_open(ctx->EL[slot], E[idx], &th);
      const int nR = count_open(ctx->ER[slot], E[idx], &th);
      all[i] = pw::make_point(E[idx], slot, nL, nR, idx, th ? 1 : 0, N, 0);
      if (th) result = PW_ETHRESH;
      else ninc = std::max(ninc, nL);
    }
    if (ninc > pw::kNlMaxOpen) return PW_EINVAL;
    const int c0 = ninc, nc = (ninc + m + 3) & ~3, ncols = 2 * n + nc;
    const size_t vec = (size_t)n * nc;
    const size_t per_pt = (nn + (size_t)n * ncols + 3 * (size_t)n) * sizeof(zc) + n * sizeof(int) +
                          (size_t)(C + K - 1) * (nn + vec) * sizeof(zc) + 2 * (size_t)(N + 2) * vec * sizeof(zc) +
                          4 * (size_t)(N + 2) * m * n * sizeof(zc) + (size_t)(N + 2) * m * m * sizeof(zc) +
                          3 * vec * sizeof(zc) + 64;
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const int fit = (int)std::max<size_t>(1, (size_t)(0.7 * (double)free_b) / per_pt);
    const int bmax = std::max(1, std::min({(int)pts.size(), 3 * ctx->num_sms, fit}));
    for (size_t b0 = 0; b0 < pts.size(); b0 += bmax) {
      const int nb = (int)std::min(pts.size() - b0, (size_t)bmax);
      std::vector<PointDesc> pd(all.begin() + b0, all.begin() + b0 + nb), loc(nb);
      for (int i = 0; i < nb; ++i) {
        pd[i] = pw::make_point(pd[i].E, pd[i].kset, pd[i].nL, pd[i].nR, pd[i].out, pd[i].skip, N, i);
        loc[i] = pd[i];
        loc[i].out = i;   // the sweep's own T goes to scratch
      }
      const size_t xs = (size_t)nb * (N + 2);
      if ((st = ensure(ctx, ctx->R, (size_t)nb * nn * sizeof(zc))) ||
          (st = ensure(ctx, ctx->M, (size_t)nb * n * ncols * sizeof(zc))) ||
          (st = ensure(ctx, ctx->piv, (size_t)nb * n * sizeof(int))) ||
          (st = ensure(ctx, ctx->KV, (size_t)nb * 3 * n * sizeof(zc))) ||
          (st = ensure(ctx, ctx->pts, (size_t)nb * sizeof(PointDesc))) ||
          (st = ensure(ctx, ctx->ptsb, (size_t)nb * sizeof(PointDesc))) ||
          (st = ensure(ctx, ctx->status, (size_t)nb * sizeof(int))) ||
          (st = ensure(ctx, ctx->Zst, (size_t)nb * C * nn * sizeof(zc))) ||
          (st = ensure(ctx, ctx->Ust, (size_t)nb * C * vec * sizeof(zc))) ||
          (K > 1 && (st = ensure(ctx, ctx->ckR, (size_t)(K - 1) * nb * nn * sizeof(zc)))) ||
          (K > 1 && (st = ensure(ctx, ctx->ckT, (size_t)(K - 1) * nb * vec * sizeof(zc)))) ||
          (st = ensure(ctx, ctx->Xa, xs * vec * sizeof(zc))) || (st = ensure(ctx, ctx->Xb, xs * vec * sizeof(zc))) ||
          (st = ensure(ctx, ctx->carry, (size_t)nb * vec * sizeof(zc))) ||
          (st = ensure(ctx, ctx->tmp, (size_t)nb * 2 * vec * sizeof(zc))) ||
          (st = ensure(ctx, ctx->Tg, (size_t)nb * sizeof(double))) ||
          (st = ensure(ctx, ctx->nlFA, xs * m * n * sizeof(zc))) || (st = ensure(ctx, ctx->nlFB, xs * m * n * sizeof(zc))) ||
          (st = ensure(ctx, ctx->nlHA, xs * m * n * sizeof(zc))) || (st = ensure(ctx, ctx->nlHB, xs * m * n * sizeof(zc))) ||
          (st = ensure(ctx, ctx->nlPP, xs * m * m * sizeof(zc))))
        return st;
      PointDesc *d_loc = (PointDesc *)ctx->pts.p, *d_pd = (PointDesc *)ctx->ptsb.p;
      CK(cudaMemcpyAsync(d_loc, loc.data(), nb * sizeof(PointDesc), cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemcpyAsync(d_pd, pd.data(), nb * sizeof(PointDesc), cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemsetAsync(ctx->status.p, 0, nb * sizeof(int), ctx->stream));
      pw::NonlocalArgs na;
      memset(&na, 0, sizeof(na));
      na.pts = d_pd;
      na.En = ctx->d_En;
      na.dz = ctx->d_dz;
      na.zedge = ctx->d_z;
      na.V = (const zc *)ctx->nlV.p;
      na.proj = ctx->d_nlproj;
      na.gl = ctx->d_gl;
      na.q = ctx->nl_q;
      na.FA = (zc *)ctx->nlFA.p;
      na.FB = (zc *)ctx->nlFB.p;
      na.HA = (zc *)ctx->nlHA.p;
      na.HB = (zc *)ctx->nlHB.p;
      na.PP = (zc *)ctx->nlPP.p;
      na.Xa = (const zc *)ctx->Xa.p;
      na.Xb = (const zc *)ctx->Xb.p;
      na.D = ctx->d_nlD;
      na.area = ctx->area;
      na.status = (const int *)ctx->status.p;
      na.T = T_dev;
      na.C = (zc *)C_dev;
      na.n = n;
      na.N = N;
      na.nc = nc;
      na.m = m;
      na.c0 = c0;
      na.ks_N = N;
      CK(pw::launch_nl_slice_terms(na, nb, ctx->stream));
      pw::SweepArgs a;
      memset(&a, 0, sizeof(a));
      a.pts = d_loc;
      a.En = ctx->d_En;
      a.O = ctx->d_O;
      a.dz = ctx->d_dz;
      a.R = ctx->R.p;
      a.M = ctx->M.p;
      a.piv = (int *)ctx->piv.p;
      a.status = (int *)ctx->status.p;
      a.T = (double *)ctx->Tg.p;
      a.n = n;
      a.N = N;
      a.nc = nc;
      a.Zst = ctx->Zst.p;
      a.Ust = ctx->Ust.p;
      a.KV = ctx->KV.p;
      a.nl_fa = (const zc *)ctx->nlFA.p;
      a.nl_fb = (const zc *)ctx->nlFB.p;
      a.nl_m = m;
      a.nl_c0 = c0;
      pw::GradArgs g;
      memset(&g, 0, sizeof(g));
      g.pts = d_loc;
      g.En = ctx->d_En;
      g.O = ctx->d_O;
      g.dz = ctx->d_dz;
      g.Zst = (const zc *)ctx->Zst.p;
      g.Ust = (const zc *)ctx->Ust.p;
      g.Xa = (zc *)ctx->Xa.p;
      g.Xb = (zc *)ctx->Xb.p;
      g.carry = (zc *)ctx->carry.p;
      g.tmp = (zc *)ctx->tmp.p;
      g.status = a.status;
      g.n = n;
      g.N = N;
      g.nc = nc;
      g.nl_fa = a.nl_fa;
      g.nl_m = m;
      g.nl_c0 = c0;
      if ((st = stored_sweep_backward(ctx, a, g, nb, C, loc, d_loc))) return st;
      CK(pw::launch_nl_solve(na, nb, ctx->stream));
      std::vector<int> sth(nb);
      CK(cudaMemcpyAsync(sth.data(), ctx->status.p, nb * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      for (int v : sth)
        if (v) result = PW_ESINGULAR;
    }
  }
  if (result == PW_ESINGULAR) latch(ctx, result);
  return result;
}

// S(0, m) of a chain of m+1 slices for npts points (FP64): the chain's modes
// U (nq = m+1 matrices) and eigenvalues En (nq x n) and thicknesses dz (nq,
// dz[0] unused) are in ctx->chU / chE / chDz; overlaps, each interface's
// S-matrix, and the star products left to right.  Result in ctx->chSa
// (npts x 4 n^2).  `pd`: npts host descriptors (E only is read; kset 0).
static pw_status chain_smatrix(pw_ctx *ctx, int nq, const std::vector<PointDesc> &pd) {
  const int n = ctx->n, npts = (int)pd.size();
  const size_t nn = (size_t)n * n, blk = (size_t)4 * nn * npts;
  pw_status st;
  if ((st = ensure(ctx, ctx->chO, (size_t)(nq - 1) * nn * sizeof(zc))) ||
      (st = ensure(ctx, ctx->chPts, (size_t)npts * sizeof(PointDesc))) ||
      (st = ensure(ctx, ctx->chSif, blk * sizeof(zc))) || (st = ensure(ctx, ctx->chSa, blk * sizeof(zc))) ||
      (st = ensure(ctx, ctx->chSb, blk * sizeof(zc))) ||
      (st = ensure(ctx, ctx->chW, (size_t)npts * 4 * nn * sizeof(zc))) ||
      (st = ensure(ctx, ctx->chPiv, (size_t)npts * n * sizeof(int))) ||
      (st = ensure(ctx, ctx->chSt, (size_t)npts * sizeof(int))))
    return st;
  CK(cudaMemcpyAsync(ctx->chPts.p, pd.data(), npts * sizeof(PointDesc), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(ctx->chSt.p, 0, npts * sizeof(int), ctx->stream));
  pw::launch_overlaps((const zc *)ctx->chU.p, (zc *)ctx->chO.p, n, nq, 1, ctx->stream, false);
  CK(cudaGetLastError());
  zc *acc = (zc *)ctx->chSa.p, *tmp = (zc *)ctx->chSb.p, *sif = (zc *)ctx->chSif.p;
  for (int q = 0; q + 1 < nq; ++q) {
    CK(pw::launch_slice_smatrix((const PointDesc *)ctx->chPts.p, (const double *)ctx->chE.p, (const zc *)ctx->chO.p,
                                (const double *)ctx->chDz.p, (zc *)ctx->chW.p, (int *)ctx->chPiv.p,
                                (int *)ctx->chSt.p, q == 0 ? acc : sif, n, nq - 2, q, npts, ctx->stream));
    if (q > 0) {
      CK(pw::launch_compose(acc, sif, tmp, (zc *)ctx->chW.p, (int *)ctx->chPiv.p, (int *)ctx->chSt.p, n, npts,
                            ctx->stream));
      std::swap(acc, tmp);
    }
  }
  if (acc != (zc *)ctx->chSa.p)
    CK(cudaMemcpyAsync(ctx->chSa.p, acc, blk * sizeof(zc), cudaMemcpyDeviceToDevice, ctx->stream));
  return PW_OK;
}

pw_status pw_set_periodic_electrode(pw_ctx *ctx, int side, int M, const pw_c128 *tables, const double *dz,
                                    const double *a3_perp) {
  if (!ctx || side < 0 || side > 1 || M < 1 || !tables || !dz || !a3_perp) return PW_EINVAL;
  if (ctx->err) return ctx->err;
  for (int q = 0; q < M; ++q)
    if (!(dz[q] > 0.0)) return PW_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->d_petab[side]) { cudaFree(ctx->d_petab[side]); ctx->d_petab[side] = nullptr; }
  ctx->pe_M[side] = 0;
  if (cudaMalloc(&ctx->d_petab[side], (size_t)M * ctx->tsz * sizeof(zc)) != cudaSuccess) {
    cudaGetLastError();
    return latch(ctx, PW_ENOMEM);
  }
  CK(cudaMemcpy(ctx->d_petab[side], tables, (size_t)M * ctx->tsz * sizeof(zc), cudaMemcpyHostToDevice));
  ctx->pe_dz[side].assign(dz, dz + M);
  ctx->pe_a3[side][0] = a3_perp[0];
  ctx->pe_a3[side][1] = a3_perp[1];
  ctx->pe_M[side] = M;
  return PW_OK;
}

pw_status pw_transmission_periodic(pw_ctx *ctx, int npts, const double *E, const double *kpar, double *T_dev) {
  if (!ctx || npts < 0 || (npts > 0 && (!E || !kpar || !T_dev)) || ctx->pe_M[0] < 1 || ctx->pe_M[1] < 1)
    return PW_EINVAL;
  if (ctx->err) return ctx->err;
  KtScope kts(ctx);
  const int n = ctx->n, N = ctx->N, ML = ctx->pe_M[0], MR = ctx->pe_M[1];
  const size_t nn = (size_t)n * n;
  const int Mmax = std::max(ML, MR);
  const int nqmax = std::max(Mmax + 1, N + 2);
  pw_status st = alloc_slots(ctx);
  if (st) return st;
  std::vector<std::vector<int>> groups;
  group_by_k(npts, kpar, groups);
  pw_status result = PW_OK;
  if ((st = ensure(ctx, ctx->peU, (size_t)(ML + MR) * nn * sizeof(zc))) ||
      (st = ensure(ctx, ctx->peV, (size_t)(ML + MR) * nn * sizeof(zc))) ||
      (st = ensure(ctx, ctx->peE, (size_t)(ML + MR) * n * sizeof(double))) ||
      (st = ensure(ctx, ctx->peStat, (size_t)(ML + MR) * sizeof(int))) ||
      (st = ensure(ctx, ctx->chU, (size_t)nqmax * nn * sizeof(zc))) ||
      (st = ensure(ctx, ctx->chE, (size_t)nqmax * n * sizeof(double))) ||
      (st = ensure(ctx, ctx->chDz, (size_t)nqmax * sizeof(double))))
    return st;
  zc *U_cell[2] = {(zc *)ctx->peU.p, (zc *)ctx->peU.p + (size_t)ML * nn};
  double *E_cell[2] = {(double *)ctx->peE.p, (double *)ctx->peE.p + (size_t)ML * n};
  for (const auto &grp : groups) {
    const double *k = kpar + 2 * grp[0];
    if ((st = ensure_ksets(ctx, std::vector<const double *>{k}))) return st;
    // modes of both electrode cells at this k_par (FP64)
    for (int side = 0; side < 2; ++side) {
      const int M = ctx->pe_M[side];
      pw::launch_assemble_h(U_cell[side], ctx->d_petab[side], ctx->d_mn, ctx->d_G, k[0], k[1], n, M, ctx->Dm,
                            ctx->Dn, ctx->stream);
      pw::launch_eig(U_cell[side], (zc *)ctx->peV.p, E_cell[side], (int *)ctx->peStat.p, n, M, ctx->stream, false);
      CK(cudaGetLastError());
    }
    const int np = (int)grp.size();
    std::vector<PointDesc> pd(np);
    std::vector<int> outs(np), bad(np, 0);
    for (int i = 0; i < np; ++i) {
      pd[i] = pw::make_point(E[grp[i]], 0, 0, 0, grp[i], 0, N, i);
      outs[i] = grp[i];
    }
    const size_t blk = (size_t)4 * nn * np;
    if ((st = ensure(ctx, ctx->bdS[0], blk * sizeof(zc))) || (st = ensure(ctx, ctx->bdS[1], blk * sizeof(zc))) ||
        (st = ensure(ctx, ctx->bdW, (size_t)np * pw::band_work_elems(n) * sizeof(zc))) ||
        (st = ensure(ctx, ctx->bdPiv, (size_t)np * 2 * n * sizeof(int))) ||
        (st = ensure(ctx, ctx->bdKeys, (size_t)np * 8 * n * sizeof(int))) ||
        (st = ensure(ctx, ctx->bdStates[0], blk * sizeof(zc))) || (st = ensure(ctx, ctx->bdStates[1], blk * sizeof(zc))) ||
        (st = ensure(ctx, ctx->bdProp[0], (size_t)np * 2 * n * sizeof(int))) ||
        (st = ensure(ctx, ctx->bdProp[1], (size_t)np * 2 * n * sizeof(int))) ||
        (st = ensure(ctx, ctx->bdStat, (size_t)2 * np * sizeof(int))) ||
        (st = ensure(ctx, ctx->bdE, (size_t)np * sizeof(double))) ||
        (st = ensure(ctx, ctx->bdBad, (size_t)np * sizeof(int))) ||
        (st = ensure(ctx, ctx->ppW, (size_t)np * pw::periodic_work_elems(n) * sizeof(zc))) ||
        (st = ensure(ctx, ctx->ppPiv, (size_t)np * 2 * n * sizeof(int))) ||
        (st = ensure(ctx, ctx->ppOut, (size_t)np * sizeof(int))))
      return st;
    std::vector<double> Eh(np);
    for (int i = 0; i < np; ++i) Eh[i] = E[grp[i]];
    CK(cudaMemcpyAsync(ctx->bdE.p, Eh.data(), np * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->ppOut.p, outs.data(), np * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    // the cells' S over one period: left [c_M, c_1' .. c_M'], right [c_1 .. c_M, c_1']
    // (primed: the next cell, its modes D U with D = diag(e^{-i G.a3_perp}))
    for (int side = 0; side < 2; ++side) {
      const int M = ctx->pe_M[side];
      zc *cu = (zc *)ctx->chU.p;
      double *ce = (double *)ctx->chE.p;
      std::vector<double> dzc(M + 1, 0.0);
      const double ax = ctx->pe_a3[side][0], ay = ctx->pe_a3[side][1];
      if (side == 0) {
        CK(cudaMemcpyAsync(cu, U_cell[0] + (size_t)(M - 1) * nn, nn * sizeof(zc), cudaMemcpyDeviceToDevice,
                           ctx->stream));
        CK(pw::launch_tilt_modes(U_cell[0], cu + nn, ctx->d_G, ax, ay, n, M, ctx->stream));
        CK(cudaMemcpyAsync(ce, E_cell[0] + (size_t)(M - 1) * n, n * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->stream));
        CK(cudaMemcpyAsync(ce + n, E_cell[0], (size_t)M * n * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->stream));
        for (int q = 0; q < M; ++q) dzc[q + 1] = ctx->pe_dz[0][q];
      } else {
        CK(cudaMemcpyAsync(cu, U_cell[1], (size_t)M * nn * sizeof(zc), cudaMemcpyDeviceToDevice, ctx->stream));
        CK(pw::launch_tilt_modes(U_cell[1], cu + (size_t)M * nn, ctx->d_G, ax, ay, n, 1, ctx->stream));
        CK(cudaMemcpyAsync(ce, E_cell[1], (size_t)M * n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ce + (size_t)M * n, E_cell[1], n * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->stream));
        for (int q = 1; q < M; ++q) dzc[q] = ctx->pe_dz[1][q];
        dzc[M] = ctx->pe_dz[1][0];
      }
      CK(cudaMemcpyAsync(ctx->chDz.p, dzc.data(), (M + 1) * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
      if ((st = chain_smatrix(ctx, M + 1, pd))) return st;
      CK(cudaMemcpyAsync(ctx->bdS[side].p, ctx->chSa.p, blk * sizeof(zc), cudaMemcpyDeviceToDevice, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));   // chDz is host-staged per side
      pw::BandArgs ba;
      ba.n = n;
      ba.nprob = np;
      ba.S = (const zc *)ctx->bdS[side].p;
      ba.Eref = E_cell[side] + (size_t)(side == 0 ? M - 1 : 0) * n;
      ba.Uref = U_cell[side] + (size_t)(side == 0 ? M - 1 : 0) * nn;
      ba.ref_shared = 1;
      ba.E = (const double *)ctx->bdE.p;
      ba.work = (zc *)ctx->bdW.p;
      ba.ipiv = (int *)ctx->bdPiv.p;
      ba.keys = (int *)ctx->bdKeys.p;
      ba.states = (zc *)ctx->bdStates[side].p;
      ba.prop = (int *)ctx->bdProp[side].p;
      ba.status = (int *)ctx->bdStat.p + (size_t)side * np;
      CK(pw::launch_cbands(ba, ctx->stream));
    }
    std::vector<int> bst(2 * np);
    CK(cudaMemcpyAsync(bst.data(), ctx->bdStat.p, 2 * np * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < np; ++i)
      if (bst[i] || bst[np + i]) { bad[i] = 1; result = PW_ENOTCONV; }
    CK(cudaMemcpyAsync(ctx->bdBad.p, bad.data(), np * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    // the device between the reference slices: [c_M (left), device slices, c_1 (right)]
    {
      zc *cu = (zc *)ctx->chU.p;
      double *ce = (double *)ctx->chE.p;
      const size_t so = 0;   // ensure_ksets put this k_par in slot 0
      CK(cudaMemcpyAsync(cu, U_cell[0] + (size_t)(ML - 1) * nn, nn * sizeof(zc), cudaMemcpyDeviceToDevice,
                         ctx->stream));
      CK(cudaMemcpyAsync(cu + nn, ctx->d_HU + (so + 1) * nn, (size_t)N * nn * sizeof(zc), cudaMemcpyDeviceToDevice,
                         ctx->stream));
      CK(cudaMemcpyAsync(cu + (size_t)(N + 1) * nn, U_cell[1], nn * sizeof(zc), cudaMemcpyDeviceToDevice,
                         ctx->stream));
      CK(cudaMemcpyAsync(ce, E_cell[0] + (size_t)(ML - 1) * n, n * sizeof(double), cudaMemcpyDeviceToDevice,
                         ctx->stream));
      CK(cudaMemcpyAsync(ce + n, ctx->d_En + (so + 1) * n, (size_t)N * n * sizeof(double), cudaMemcpyDeviceToDevice,
                         ctx->stream));
      CK(cudaMemcpyAsync(ce + (size_t)(N + 1) * n, E_cell[1], n * sizeof(double), cudaMemcpyDeviceToDevice,
                         ctx->stream));
      std::vector<double> dzc(N + 2, 0.0);
      for (int q = 1; q <= N; ++q) dzc[q] = ctx->dz[q];
      dzc[N + 1] = ctx->pe_dz[1][0];
      CK(cudaMemcpyAsync(ctx->chDz.p, dzc.data(), (N + 2) * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
      if ((st = chain_smatrix(ctx, N + 2, pd))) return st;
      CK(cudaStreamSynchronize(ctx->stream));
    }
    pw::PeriodicArgs pa;
    pa.n = n;
    pa.Sdev = (const zc *)ctx->chSa.p;
    pa.statesL = (const zc *)ctx->bdStates[0].p;
    pa.statesR = (const zc *)ctx->bdStates[1].p;
    pa.propL = (const int *)ctx->bdProp[0].p;
    pa.propR = (const int *)ctx->bdProp[1].p;
    pa.bad = (const int *)ctx->bdBad.p;
    pa.work = (zc *)ctx->ppW.p;
    pa.ipiv = (int *)ctx->ppPiv.p;
    pa.T = T_dev;
    pa.out = (const int *)ctx->ppOut.p;
    CK(pw::launch_periodic_solve(pa, np, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if (result != PW_OK) latch(ctx, result);
  return result;
}

pw_status pw_set_grad_checkpoint(pw_ctx *ctx, int interval) {
  if (!ctx || interval < 0) return PW_EINVAL;
  ctx->grad_interval = interval;
  return PW_OK;
}

pw_status pw_workspace_bytes(const pw_ctx *ctx, double *bytes) {
  if (!ctx || !bytes) return PW_EINVAL;
  const DevBuf *b[] = {&ctx->R, &ctx->M, &ctx->piv, &ctx->pts, &ctx->status, &ctx->work, &ctx->KV,
                       &ctx->rowexp, &ctx->Zst, &ctx->Ust, &ctx->LUst, &ctx->PIVst, &ctx->Xa, &ctx->Xb,
                       &ctx->Fr, &ctx->Gr, &ctx->carry, &ctx->tmp, &ctx->Xa_m, &ctx->Xb_m, &ctx->status_m,
                       &ctx->Tg, &ctx->Gam, &ctx->gtab, &ctx->T1, &ctx->dV0, &ctx->wgt, &ctx->corr,
                       &ctx->eigws, &ctx->bw, &ctx->dshift, &ctx->lead_scr, &ctx->lead_out, &ctx->ckR,
                       &ctx->ckT};
  double t = 0.0;
  for (const DevBuf *x : b) t += (double)x->bytes;
  *bytes = t;
  return PW_OK;
}

pw_status pw_grad(pw_ctx *ctx, int npts, const double *E, const double *kpar, const double *weight,
                  double *sumT_host, double *dV0_host, double *dgap_host) {
  if (!ctx || npts < 0 || (npts > 0 && (!E || !kpar)) || !sumT_host) return PW_EINVAL;
  if (ctx->err) return ctx->err;
  KtScope kts(ctx);
  if (dgap_host && !ctx->has_shift) return PW_EINVAL;   // no geometry motion was given
  if (dV0_host && ctx->n_wells == 0) return PW_EINVAL;   // explicit tables have no wells
  const bool lead_shift = dgap_host && (ctx->lead_rate[0][0] != 0.0 || ctx->lead_rate[0][1] != 0.0 ||
                                        ctx->lead_rate[1][0] != 0.0 || ctx->lead_rate[1][1] != 0.0);
  double dgap_sum = 0.0;
  const int n = ctx->n, N = ctx->N;
  const size_t nn = (size_t)n * n;
  const int tsz = ctx->tsz;
  pw_status st = alloc_slots(ctx);
  if (st) return st;
  // Gamma_p and the fold's scratch for one chunk of C device slices
  const int C = grad_interval_of(ctx);
  if ((st = ensure(ctx, ctx->Gam, (size_t)C * nn * sizeof(zc))) ||
      (st = ensure(ctx, ctx->gtab, (size_t)N * tsz * sizeof(zc))) ||
      (st = ensure(ctx, ctx->T1, (size_t)C * nn * sizeof(zc))) ||
      (st = ensure(ctx, ctx->dV0, (size_t)std::max(1, ctx->n_wells) * sizeof(double))))
    return st;
  CK(cudaMemsetAsync(ctx->gtab.p, 0, (size_t)N * tsz * sizeof(zc), ctx->stream));
  std::vector<std::vector<int>> groups;
  group_by_k(npts, kpar, groups);
  double sumT = 0.0;
  pw_status result = PW_OK;
  for (size_t g0 = 0; g0 < groups.size(); g0 += ctx->ks_cap) {
    const size_t g1 = std::min(groups.size(), g0 + (size_t)ctx->ks_cap);
    std::vector<const double *> ks;
    std::vector<std::pair<int, int>> pts;
    for (size_t gi = g0; gi < g1; ++gi) {
      ks.push_back(kpar + 2 * groups[gi][0]);
      for (int idx : groups[gi]) pts.emplace_back(idx, (int)(gi - g0));
    }
    if ((st = ensure_ksets(ctx, ks))) return st;
    std::vector<PointDesc> all(pts.size());
    int nc = 1;
    for (size_t i = 0; i < pts.size(); ++i) {
      const int idx = pts[i].first, slot = pts[i].second;
      bool th = false;
      const int nL = count_open(ctx->EL[slot], E[idx], &th);
      const int nR = count_open(ctx->ER[slot], E[idx], &th);
      all[i] = pw::make_point(E[idx], slot, nL, nR, idx, th ? 1 : 0, N, 0);
      if (th) result = PW_ETHRESH;
      else nc = std::max(nc, std::max(nL, nR));
    }
    nc = (nc + 3) & ~3;
    const int ncols = 2 * n + nc;
    const size_t vec = (size_t)n * nc;
    // checkpointed recomputation: the sweep state (R, Tacc) is kept at the start
    // of every segment of C interfaces, and Z_p, u_p only for the C interfaces of
    // the segment being recomputed, so the stores grow as (ceil((N+1)/C) - 1 + C)
    // (n^2 + n nc), about 2 sqrt(N+1) (n^2 + n nc) for C = ceil(sqrt(N+1))
    const int K = (N + 1 + C - 1) / C;   // segments
    // per point: FP64 sweep buffers, the stores of one segment, the checkpoints,
    // amplitudes of both problems
    const size_t per_pt = (nn + (size_t)n * ncols + 3 * (size_t)n) * sizeof(zc) + n * sizeof(int) +
                          (size_t)C * (nn + vec) * sizeof(zc) + (size_t)(K - 1) * (nn + vec) * sizeof(zc) +
                          4 * (size_t)(N + 2) * vec * sizeof(zc) + 3 * vec * sizeof(zc) + 64;
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const size_t have = free_b + ctx->R.bytes + ctx->M.bytes + ctx->Zst.bytes + ctx->Ust.bytes +
                        ctx->Xa.bytes + ctx->Xb.bytes + ctx->Xa_m.bytes + ctx->Xb_m.bytes + ctx->ckR.bytes +
                        ctx->ckT.bytes;
    const int fit = (int)std::max<size_t>(1, (size_t)(0.8 * (double)have) / per_pt);
    const int bmax = std::max(1, std::min({(int)pts.size(), 3 * ctx->num_sms, fit}));
    for (size_t b0 = 0; b0 < pts.size(); b0 += bmax) {
      const int nb = (int)std::min(pts.size() - b0, (size_t)bmax);
      std::vector<PointDesc> pd(all.begin() + b0, all.begin() + b0 + nb);
      for (int i = 0; i < nb; ++i) pd[i] = pw::make_point(pd[i].E, pd[i].kset, pd[i].nL, pd[i].nR, pd[i].out,
                                                          pd[i].skip, N, i);
      std::vector<PointDesc> pm(pd);
      for (auto &q : pm) std::swap(q.nL, q.nR);     // mirrored: incident from the right electrode
      std::vector<double> w(nb, 1.0);
      if (weight)
        for (int i = 0; i < nb; ++i) w[i] = weight[pd[i].out];
      if ((st = ensure(ctx, ctx->R, (size_t)nb * nn * sizeof(zc))) ||
          (st = ensure(ctx, ctx->M, (size_t)nb * n * ncols * sizeof(zc))) ||
          (st = ensure(ctx, ctx->piv, (size_t)nb * n * sizeof(int))) ||
          (st = ensure(ctx, ctx->KV, (size_t)nb * 3 * n * sizeof(zc))) ||
          (st = ensure(ctx, ctx->pts, (size_t)2 * nb * sizeof(PointDesc))) ||
          (st = ensure(ctx, ctx->status, (size_t)nb * sizeof(int))) ||
          (st = ensure(ctx, ctx->status_m, (size_t)nb * sizeof(int))) ||
          (st = ensure(ctx, ctx->Zst, (size_t)nb * C * nn * sizeof(zc))) ||
          (st = ensure(ctx, ctx->Ust, (size_t)nb * C * vec * sizeof(zc))) ||
          (K > 1 && (st = ensure(ctx, ctx->ckR, (size_t)(K - 1) * nb * nn * sizeof(zc)))) ||
          (K > 1 && (st = ensure(ctx, ctx->ckT, (size_t)(K - 1) * nb * vec * sizeof(zc)))) ||
          (st = ensure(ctx, ctx->Xa, (size_t)nb * (N + 2) * vec * sizeof(zc))) ||
          (st = ensure(ctx, ctx->Xb, (size_t)nb * (N + 2) * vec * sizeof(zc))) ||
          (st = ensure(ctx, ctx->Xa_m, (size_t)nb * (N + 2) * vec * sizeof(zc))) ||
          (st = ensure(ctx, ctx->Xb_m, (size_t)nb * (N + 2) * vec * sizeof(zc))) ||
          (st = ensure(ctx, ctx->carry, (size_t)nb * vec * sizeof(zc))) ||
          (st = ensure(ctx, ctx->tmp, (size_t)nb * 2 * vec * sizeof(zc))) ||
          (st = ensure(ctx, ctx->Tg, (size_t)2 * nb * sizeof(double))) ||
          (st = ensure(ctx, ctx->wgt, (size_t)nb * sizeof(double))))
        return st;
      PointDesc *d_pd = (PointDesc *)ctx->pts.p, *d_pm = d_pd + nb;
      CK(cudaMemcpyAsync(d_pd, pd.data(), nb * sizeof(PointDesc), cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemcpyAsync(d_pm, pm.data(), nb * sizeof(PointDesc), cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemcpyAsync(ctx->wgt.p, w.data(), nb * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemsetAsync(ctx->status.p, 0, nb * sizeof(int), ctx->stream));
      CK(cudaMemsetAsync(ctx->status_m.p, 0, nb * sizeof(int), ctx->stream));
      // outputs of the two sweeps: T of the original, unused T of the mirrored
      // problem (each point writes slot `out` - remap to the batch index)
      std::vector<PointDesc> pd_local(pd), pm_local(pm);
      for (int i = 0; i < nb; ++i) { pd_local[i].out = i; pm_local[i].out = nb + i; }
      CK(cudaMemcpyAsync(d_pd, pd_local.data(), nb * sizeof(PointDesc), cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemcpyAsync(d_pm, pm_local.data(), nb * sizeof(PointDesc), cudaMemcpyHostToDevice, ctx->stream));
      for (int mirror = 0; mirror < 2; ++mirror) {
        std::vector<PointDesc> &loc = mirror ? pm_local : pd_local;
        PointDesc *d_loc = mirror ? d_pm : d_pd;
        pw::SweepArgs a;
        memset(&a, 0, sizeof(a));
        a.pts = mirror ? d_pm : d_pd;
        a.En = ctx->d_En;
        a.O = ctx->d_O;
        a.dz = ctx->d_dz;
        a.R = ctx->R.p;
        a.M = ctx->M.p;
        a.piv = (int *)ctx->piv.p;
        a.status = (int *)(mirror ? ctx->status_m.p : ctx->status.p);
        a.T = (double *)ctx->Tg.p;
        a.n = n;
        a.N = N;
        a.nc = nc;
        a.Zst = ctx->Zst.p;
        a.Ust = ctx->Ust.p;
        a.KV = ctx->KV.p;
        a.mirror = mirror;
        pw::GradArgs g;
        g.pts = a.pts;
        g.En = ctx->d_En;
        g.O = ctx->d_O;
        g.dz = ctx->d_dz;
        g.Zst = (const zc *)ctx->Zst.p;
        g.Ust = (const zc *)ctx->Ust.p;
        g.Xa = (zc *)(mirror ? ctx->Xa_m.p : ctx->Xa.p);
        g.Xb = (zc *)(mirror ? ctx->Xb_m.p : ctx->Xb.p);
        g.carry = (zc *)ctx->carry.p;
        g.tmp = (zc *)ctx->tmp.p;
        g.status = a.status;
        g.n = n;
        g.N = N;
        g.nc = nc;
        g.mirror = mirror;
        g.nl_fa = nullptr;
        g.nl_m = 0;
        g.nl_c0 = 0;
        if ((st = stored_sweep_backward(ctx, a, g, nb, C, loc, d_loc))) return st;
      }
      pw::GammaArgs h;
      h.pts = d_pd;
      h.En = ctx->d_En;
      h.dz = ctx->d_dz;
      h.Xa = (const zc *)ctx->Xa.p;
      h.Xb = (const zc *)ctx->Xb.p;
      h.Xa_m = (const zc *)ctx->Xa_m.p;
      h.Xb_m = (const zc *)ctx->Xb_m.p;
      h.status = (const int *)ctx->status.p;
      h.status_m = (const int *)ctx->status_m.p;
      h.weight = (const double *)ctx->wgt.p;
      h.Gam = (zc *)ctx->Gam.p;
      h.gtab = (zc *)ctx->gtab.p;
      h.n = n;
      h.N = N;
      h.nc = nc;
      h.npts = nb;
      // Gamma_p of this batch's points, folded onto the tables' grid chunk by
      // chunk of C slices (the fold is linear, so batches add up in gtab)
      for (size_t sl = 0; sl < ks.size(); ++sl)
        for (int p0 = 1; p0 <= N; p0 += C) {
          const int cnt = std::min(C, N + 1 - p0);
          CK(cudaMemsetAsync(ctx->Gam.p, 0, (size_t)cnt * nn * sizeof(zc), ctx->stream));
          CK(pw::launch_grad_gamma(h, (int)sl, p0, cnt, ctx->stream));
          CK(pw::launch_grad_fold(h, (int)sl, p0, cnt, ctx->d_HU, (zc *)ctx->T1.p, ctx->d_mn, ctx->Dm,
                                  ctx->Dn, ctx->stream));
        }
      std::vector<double> lead_h(nb, 0.0);
      if (lead_shift) {
        if ((st = ensure(ctx, ctx->lead_scr, (size_t)nb * 4 * vec * sizeof(zc))) ||
            (st = ensure(ctx, ctx->lead_out, (size_t)nb * sizeof(double))))
          return st;
        CK(pw::launch_grad_leads(h, ctx->d_HU, ctx->d_G, (zc *)ctx->lead_scr.p, ctx->lead_rate,
                                 (double *)ctx->lead_out.p, ctx->stream));
        CK(cudaMemcpyAsync(lead_h.data(), ctx->lead_out.p, nb * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream));
      }
      std::vector<double> Th(nb);
      std::vector<int> sth(nb), stm(nb);
      CK(cudaMemcpyAsync(Th.data(), ctx->Tg.p, nb * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaMemcpyAsync(sth.data(), ctx->status.p, nb * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaMemcpyAsync(stm.data(), ctx->status_m.p, nb * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      for (int i = 0; i < nb; ++i) {
        if (sth[i] || stm[i]) result = PW_ESINGULAR;
        else if (!pd[i].skip) {
          sumT += w[i] * Th[i];
          dgap_sum += w[i] * lead_h[i];
        }
      }
    }
  }
  *sumT_host = sumT;
  const bool wells_shift = dgap_host && ctx->d_wrate && ctx->n_wells > 0;
  if (dV0_host || wells_shift) {
    if (wells_shift && (st = ensure(ctx, ctx->dshift, (size_t)ctx->n_wells * sizeof(double)))) return st;
    pw::GammaArgs h;
    memset(&h, 0, sizeof(h));
    h.gtab = (zc *)ctx->gtab.p;
    h.n = n;
    h.N = N;
    pw::WellSet ws;
    ws.xyz = ctx->d_wxyz;
    ws.v0 = ctx->d_wv0;
    ws.sigma = ctx->d_wsig;
    ws.n = ctx->n_wells;
    const double b[4] = {ctx->b1[0], ctx->b1[1], ctx->b2[0], ctx->b2[1]};
    CK(pw::launch_grad_wells(h, ws, ctx->d_z, b, ctx->area, ctx->Dm, ctx->Dn,
                             dV0_host ? (double *)ctx->dV0.p : nullptr, wells_shift ? ctx->d_wrate : nullptr,
                             wells_shift ? (double *)ctx->dshift.p : nullptr, ctx->stream));
    if (dV0_host)
      CK(cudaMemcpyAsync(dV0_host, ctx->dV0.p, ctx->n_wells * sizeof(double), cudaMemcpyDeviceToHost,
                         ctx->stream));
    std::vector<double> sh(wells_shift ? ctx->n_wells : 0);
    if (wells_shift)
      CK(cudaMemcpyAsync(sh.data(), ctx->dshift.p, ctx->n_wells * sizeof(double), cudaMemcpyDeviceToHost,
                         ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (double v : sh) dgap_sum += v;
  }
  if (dgap_host) *dgap_host = dgap_sum;
  if (result == PW_ESINGULAR) latch(ctx, result);
  return result;
}

}  // extern "C"
